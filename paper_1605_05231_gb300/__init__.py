"""GB300-native radial-line 3D NUFFT projector (forward + adjoint)."""
