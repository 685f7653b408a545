// Batches of independent projector problems of mixed sizes.  A batch owns one
// plan per item.  Its forward + adjoint over all items is captured once into a
// CUDA graph: items are dealt, largest first, to the least loaded of up to 12
// worker streams forked from the caller's stream, so small problems run
// concurrently, and every later call
// replays the whole sequence with one cudaGraphLaunch.  The graph is captured
// again only when the caller passes different buffers.
#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

struct nufft3d_batch_s {
  std::vector<nufft3d_plan> plans;
  bool grouping = false;                  // grouped interpolation launches (see capture)
  std::vector<nufft::GroupItem*> d_items;  // per group of the last capture, device copies
  std::vector<int*> d_counters;           // per group: the spread's work counter
  std::vector<cudaEvent_t> evs;           // events of the last capture
  int device = 0;
  cudaStream_t cap = nullptr;  // capture origin (the legacy stream cannot be captured)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  std::vector<cudaStream_t> gstreams;  // one per group of the last capture (kept for reuse)
  std::vector<cudaEvent_t> gjoin;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;  // buffers the graph was captured with
};

namespace {

constexpr int kMaxWorkerStreams = 12;

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  return e == cudaErrorMemoryAllocation ? NUFFT3D_ERR_NOMEM : NUFFT3D_ERR_CUDA;
}

void free_capture_resources(nufft3d_batch b) {
  for (auto* p : b->d_items) cudaFree(p);
  for (auto* p : b->d_counters) cudaFree(p);
  for (cudaEvent_t e : b->evs) cudaEventDestroy(e);
  b->d_items.clear();
  b->d_counters.clear();
  b->evs.clear();
}

void free_batch(nufft3d_batch b) {
  if (!b) return;
  free_capture_resources(b);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaStream_t s : b->gstreams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->gjoin) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (nufft3d_plan p : b->plans) nufft3d_plan_destroy(p);
  delete b;
}

// A plan whose interpolation can join a group launch: exact coefficients with
// the scheduled gather (10) and the real-weight spread (7) on complex64 grids.
bool groupable(const nufft3d_plan p) {
  return p->real_ok && p->sched_ok && p->gather_variant == 10 && p->spread_variant == 7 &&
         p->grid_dtype == NUFFT3D_GRID_C64 && p->T == 8 && p->J == 6 && p->pts_per_sub <= 256;
}

nufft::GroupItem group_item(const nufft3d_plan p, void* lines) {
  nufft::GroupItem it{};
  it.pg = nufft::PointGeom{p->K, p->M, p->d_dir, p->d_rad};
  it.sorted = p->d_sorted;
  it.subs = p->d_sub;
  it.n_subs = p->n_sub;
  it.sched = p->d_sched;
  it.gslots = p->d_gslots;
  it.box = p->d_box;
  it.err = p->d_err;
  it.grid = p->d_grid;
  it.lines = (float2*)lines;
  it.adj_in = p->do_line_fft ? p->d_lines : (const float2*)lines;
  it.adj_grid = p->d_grid_adj;
  return it;
}

// The whole forward + adjoint of every item, recorded as one CUDA graph.
// Plans that share N, K and J (and run the default exact-coefficient kernels)
// form groups of up to kMaxGroupItems: their FFT passes and line DFTs run per
// plan on the worker streams, but their interpolation is one launch per group
// for the gather and one persistent launch for the spread, whose CTAs pull
// (plan, subproblem) work items from a single counter.  Other plans run their
// whole sequence on a worker stream.
int capture(nufft3d_batch b, const void* const* vols, void* const* lines, void* const* vols_out,
            cudaStream_t launch_st) {
  const int n = (int)b->plans.size();
  cudaStream_t st = b->cap;
  const int ns = (int)b->streams.size();
  free_capture_resources(b);
  // groups
  std::vector<std::vector<int>> groups;
  std::vector<int> single;
  {
    std::vector<bool> used(n, false);
    for (int i = 0; i < n; ++i) {
      if (used[i]) continue;
      const nufft3d_plan p = b->plans[i];
      if (!b->grouping || !groupable(p)) {
        single.push_back(i);
        continue;
      }
      std::vector<int> grp{i};
      used[i] = true;
      for (int k = i + 1; k < n && (int)grp.size() < nufft::kMaxGroupItems; ++k) {
        const nufft3d_plan q = b->plans[k];
        if (!used[k] && groupable(q) && q->N == p->N && q->K == p->K && q->J == p->J) {
          grp.push_back(k);
          used[k] = true;
        }
      }
      if (grp.size() == 1) {
        single.push_back(i);
      } else {
        groups.push_back(grp);
      }
    }
  }
  // the group tables, uploaded before the capture
  std::vector<nufft::GroupParams> gps(groups.size());
  cudaError_t e = cudaSuccess;
  for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
    const auto& grp = groups[gi];
    const nufft3d_plan p0 = b->plans[grp[0]];
    nufft::GroupParams& gp = gps[gi];
    gp = nufft::GroupParams{};
    gp.rpoly = p0->rpoly;
    gp.K = p0->K;
    gp.nT = p0->nT;
    gp.n_items = (int)grp.size();
    std::vector<nufft::GroupItem> items;
    int acc = 0;
    for (size_t k = 0; k < grp.size(); ++k) {
      gp.work_begin[k] = acc;
      acc += b->plans[grp[k]]->n_sub;
      items.push_back(group_item(b->plans[grp[k]], lines[grp[k]]));
    }
    gp.work_begin[grp.size()] = acc;
    nufft::GroupItem* d = nullptr;
    int* c = nullptr;
    e = cudaMalloc((void**)&d, items.size() * sizeof(nufft::GroupItem));
    if (e == cudaSuccess) b->d_items.push_back(d);
    if (e == cudaSuccess) e = cudaMemcpy(d, items.data(), items.size() * sizeof(nufft::GroupItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c, sizeof(int));
    if (e == cudaSuccess) b->d_counters.push_back(c);
  }
  // a stream and a join event per group, made before the capture
  for (size_t gi = b->gstreams.size(); gi < groups.size() && e == cudaSuccess; ++gi) {
    cudaStream_t gst;
    cudaEvent_t gev;
    e = cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->gstreams.push_back(gst);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->gjoin.push_back(gev);
  }
  if (e != cudaSuccess) return cuda_rc(e);
  auto new_event = [&](cudaEvent_t* ev) {
    cudaError_t r = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (r == cudaSuccess) b->evs.push_back(*ev);
    return r;
  };
  e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_rc(e);
  int rc = NUFFT3D_OK;
  e = cudaEventRecord(b->fork, st);
  for (int s = 0; s < ns && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->streams[s], b->fork, 0);
  // the groups, stage by stage across groups (so that no group's later stage
  // sits in a worker stream's queue ahead of another group's earlier stage):
  // items dealt round-robin over the worker streams, each group's two
  // interpolation launches on a group stream of its own
  std::vector<double> load(ns, 0.0);
  auto work = [&](int i) {
    const nufft3d_plan p = b->plans[i];
    return (double)p->P_eval + (double)p->K * p->K * p->K;
  };
  const size_t ng = groups.size();
  for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi) e = cudaStreamWaitEvent(b->gstreams[gi], b->fork, 0);
  std::vector<std::vector<cudaStream_t>> ws(ng);
  {
    int next = 0;
    for (size_t gi = 0; gi < ng; ++gi)
      for (int i : groups[gi]) {
        ws[gi].push_back(b->streams[next]);
        load[next] += work(i);
        next = (next + 1) % ns;
      }
  }
  // each group's per-item stage `part` on the worker streams, then the group
  // stream waits for all of them
  auto stage = [&](size_t gi, cudaEvent_t after, auto&& body) {
    const auto& grp = groups[gi];
    for (size_t j = 0; j < grp.size() && rc == NUFFT3D_OK && e == cudaSuccess; ++j) {
      if (after) e = cudaStreamWaitEvent(ws[gi][j], after, 0);
      if (e != cudaSuccess) break;
      rc = body(b->plans[grp[j]], grp[j], ws[gi][j]);
      cudaEvent_t ev;
      if (rc == NUFFT3D_OK) e = new_event(&ev);
      if (e == cudaSuccess) e = cudaEventRecord(ev, ws[gi][j]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->gstreams[gi], ev, 0);
    }
  };
  std::vector<cudaEvent_t> g1(ng, nullptr), g2(ng, nullptr);
  // stage 1: everything before the gather, per plan
  for (size_t gi = 0; gi < ng; ++gi)
    stage(gi, nullptr, [&](nufft3d_plan p, int i, cudaStream_t w) {
      return nufft::plan_forward_parts(p, vols[i], lines[i], w, 1);
    });
  for (size_t gi = 0; gi < ng && e == cudaSuccess && rc == NUFFT3D_OK; ++gi) {
    e = nufft::launch_group_gather(gps[gi], b->d_items[gi], b->gstreams[gi]);
    if (e == cudaSuccess) e = new_event(&g1[gi]);
    if (e == cudaSuccess) e = cudaEventRecord(g1[gi], b->gstreams[gi]);
  }
  // stage 2: the forward line DFTs and the adjoint line DFTs, per plan
  for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi)
    stage(gi, g1[gi], [&](nufft3d_plan p, int i, cudaStream_t w) {
      int r = nufft::plan_forward_parts(p, vols[i], lines[i], w, 4);
      if (r == NUFFT3D_OK) r = nufft::plan_adjoint_parts(p, lines[i], vols_out[i], w, 1);
      return r;
    });
  for (size_t gi = 0; gi < ng && e == cudaSuccess && rc == NUFFT3D_OK; ++gi) {
    e = nufft::launch_group_spread(gps[gi], b->d_items[gi], b->d_counters[gi], b->gstreams[gi]);
    if (e == cudaSuccess) e = new_event(&g2[gi]);
    if (e == cudaSuccess) e = cudaEventRecord(g2[gi], b->gstreams[gi]);
  }
  // stage 3: the inverse FFT passes, per plan
  for (size_t gi = 0; gi < ng && e == cudaSuccess && rc == NUFFT3D_OK; ++gi) {
    const auto& grp = groups[gi];
    for (size_t j = 0; j < grp.size() && rc == NUFFT3D_OK && e == cudaSuccess; ++j) {
      e = cudaStreamWaitEvent(ws[gi][j], g2[gi], 0);
      if (e == cudaSuccess)
        rc = nufft::plan_adjoint_parts(b->plans[grp[j]], lines[grp[j]], vols_out[grp[j]], ws[gi][j], 4);
    }
  }
  for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi) {
    e = cudaEventRecord(b->gjoin[gi], b->gstreams[gi]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->gjoin[gi], 0);
  }
  // the other items: largest first to the least loaded worker stream (work
  // taken as the evaluated points plus the grid cells)
  std::stable_sort(single.begin(), single.end(), [&](int a, int c) { return work(a) > work(c); });
  for (size_t q = 0; q < single.size() && e == cudaSuccess && rc == NUFFT3D_OK; ++q) {
    const int i = single[q];
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += work(i);
    cudaStream_t ws = b->streams[w];
    rc = nufft::plan_forward_enqueue(b->plans[i], vols[i], lines[i], ws);
    if (rc == NUFFT3D_OK) rc = nufft::plan_adjoint_enqueue(b->plans[i], lines[i], vols_out[i], ws);
  }
  for (int s = 0; s < ns && e == cudaSuccess; ++s) {
    e = cudaEventRecord(b->join[s], b->streams[s]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[s], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = e2;
  if (rc != NUFFT3D_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != NUFFT3D_OK ? rc : cuda_rc(e);
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_rc(e);
  }
  for (nufft3d_plan p : b->plans) p->last_stream = launch_st;
  return NUFFT3D_OK;
}

}  // namespace

extern "C" {

int nufft3d_batch_create(nufft3d_batch* out, const nufft3d_params* ps, int count, void* cuda_stream) {
  if (!out) return NUFFT3D_ERR_ARG;
  *out = nullptr;
  if (!ps || count < 1) return NUFFT3D_ERR_ARG;
  nufft3d_batch b = new (std::nothrow) nufft3d_batch_s();
  if (!b) return NUFFT3D_ERR_NOMEM;
  int rc = NUFFT3D_OK;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) rc = cuda_rc(e);
  for (int i = 0; i < count && rc == NUFFT3D_OK; ++i) {
    nufft3d_plan p = nullptr;
    rc = nufft3d_plan_create(&p, ps + i, cuda_stream);
    if (rc == NUFFT3D_OK) b->plans.push_back(p);
  }
  const int ns = count < kMaxWorkerStreams ? count : kMaxWorkerStreams;
  for (int s = 0; s < ns && rc == NUFFT3D_OK; ++s) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
    if (e != cudaSuccess) rc = cuda_rc(e);
  }
  if (rc == NUFFT3D_OK) {
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_rc(e);
  }
  if (rc != NUFFT3D_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return NUFFT3D_OK;
}

int nufft3d_batch_size(nufft3d_batch b, int* count) {
  if (!b || !count) return NUFFT3D_ERR_ARG;
  *count = (int)b->plans.size();
  return NUFFT3D_OK;
}

int nufft3d_batch_item(nufft3d_batch b, int i, nufft3d_plan* out) {
  if (!b || !out || i < 0 || i >= (int)b->plans.size()) return NUFFT3D_ERR_ARG;
  *out = b->plans[i];
  return NUFFT3D_OK;
}

int nufft3d_batch_forward_adjoint(nufft3d_batch b, const void* const* vols, void* const* lines,
                                  void* const* vols_out, void* cuda_stream) {
  if (!b || !vols || !lines || !vols_out) return NUFFT3D_ERR_ARG;
  const int n = (int)b->plans.size();
  std::vector<const void*> key;
  key.reserve(3 * n);
  for (int i = 0; i < n; ++i) {
    if (!vols[i] || !lines[i] || !vols_out[i]) return NUFFT3D_ERR_ARG;
    key.push_back(vols[i]);
    key.push_back(lines[i]);
    key.push_back(vols_out[i]);
  }
  nufft::DeviceGuard guard(b->device);
  if (guard.status != cudaSuccess) return cuda_rc(guard.status);
  cudaError_t e = cudaSuccess;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!b->exec || key != b->key) {
    // plans' earlier work on other streams must not race the replay
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_rc(e);
    const int rc = capture(b, vols, lines, vols_out, st);
    if (rc != NUFFT3D_OK) return rc;
    b->key = key;
  }
  return cuda_rc(cudaGraphLaunch(b->exec, st));
}

int nufft3d_batch_set_grouping(nufft3d_batch b, int on) {
  if (!b) return NUFFT3D_ERR_ARG;
  b->grouping = on != 0;
  b->key.clear();
  return NUFFT3D_OK;
}

int nufft3d_batch_invalidate(nufft3d_batch b) {
  if (!b) return NUFFT3D_ERR_ARG;
  b->key.clear();
  return NUFFT3D_OK;
}

int nufft3d_batch_destroy(nufft3d_batch b) {
  if (!b) return NUFFT3D_OK;
  nufft::DeviceGuard guard(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
  return NUFFT3D_OK;
}

}  // extern "C"
