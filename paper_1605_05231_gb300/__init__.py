"""GB300-native radial-line 3D NUFFT projector (forward + adjoint).

The compute runs in libnufft3d.so (hand-written CUDA for sm_103a) behind the
C ABI of include/nufft3d.h; ``binding`` marshals torch tensors to it.
"""
from .binding import (Batch, HostPipeline, Plan, PolarNufft, ReverseGrangeat, NufftError, fourier_slice_weights, load_library,  # noqa: F401
                      polar_resample, project, workspace_bytes, fp32_fma_peak)
