// wf_batch.cu -- batched solves of many independent maps of uneven sizes.
//
// Each map has its own plan (workspace, graphs, private stream).  The maps
// are spread over L lanes: a lane is a host worker thread with its own CUDA
// stream that runs its maps' wf_solve one after another.  Up to L solves are
// then in flight on the GPU at once, which is what small maps need: a 256 x
// 256 map gives a column pass of only 16 CTAs and a row pass of 256, far
// from the 152 SMs the GPU has, and the launch-bound iteration of one map
// leaves the SMs idle between its kernels.  Nothing is shared between the
// lanes but the device, so a map's result is bit for bit the one wf_solve
// gives for it alone.
//
// Lane assignment: largest map first, each to the lane with the fewest
// pixels so far (LPT on pixels; every map runs the same schedule, so pixels
// stand in for its cost).
//
// Persistent mode (lanes = 0): the maps' sweeps run together in one
// persistent cooperative launch per residual checkpoint (wf_batchk.cu: device
// work queues over (map, row group) and (map, column group) items, grid
// barriers between the phases, per-map done flags), captured with every
// map's residual and controller kernels in one CUDA graph per polling chunk.
// The other steps of a solve -- loading, the defect corrections' residuals
// and sources, the output -- are wf_solve's own (SolveJob), taken for all
// maps between the runs.  A tuner times the two compiled shapes of each size
// on the first map of that size and keeps the faster, per size and device,
// for the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/wf.h"
#include "wf_internal.h"

struct wf_batch_s {
  int nmaps = 0;
  int lanes = 0;
  int device = 0;
  bool persistent = false;    // lanes = 0
  cudaStream_t pstream = nullptr;
  cudaEvent_t ev_out = nullptr;
  wf::BatchDevice bd;
  std::vector<void*> dev_allocs;
  std::vector<int> ny, nx;
  std::vector<wf_plan_t> plans;
  std::vector<std::vector<int>> lane_maps;
  std::vector<cudaStream_t> lane_stream;
  std::vector<cudaEvent_t> lane_done;
  cudaEvent_t ev_in = nullptr;
  cudaStream_t user = nullptr;
};

namespace {

constexpr int kMaxMaps = 65536;
constexpr int kMaxLanes = 64;
constexpr int kNotRun = -1;

void destroy(wf_batch_s* B) {
  for (wf_plan_t p : B->plans)
    if (p) wf_plan_destroy(p);
  for (void* q : B->dev_allocs) cudaFree(q);
  if (B->pstream) cudaStreamDestroy(B->pstream);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  for (cudaEvent_t e : B->lane_done)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : B->lane_stream)
    if (s) cudaStreamDestroy(s);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  delete B;
}

// shape (0 or 1) per map size and device, chosen by timing
std::mutex g_shape_mu;
std::map<std::pair<int, int>, int> g_shape;

template <class T>
bool dalloc(wf_batch_s* B, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  B->dev_allocs.push_back(q);
  *p = (T*)q;
  return true;
}

// what the persistent kernel takes (host only, before any CUDA call)
int check_persistent(int nmaps, const int* ny, const int* nx, unsigned parts, const wf_params* p) {
  wf_params prm;
  if (p) prm = *p;
  else wf_params_default(&prm);
  if (!(parts & WF_PART_STRIPE) || ((parts & WF_PART_1F) && !prm.merge_2df) || prm.dft_precision != 0)
    return WF_EUNSUPPORTED;
  for (int i = 0; i < nmaps; ++i)
    if (ny[i] != nx[i] || wf::batch_class(ny[i], 0) < 0) return WF_EUNSUPPORTED;
  return WF_OK;
}

int create_persistent(wf_batch_s* B, unsigned parts, const wf_params* p) {
  wf_params prm;
  if (p) prm = *p;
  else wf_params_default(&prm);
  size_t cap = 0;
  for (int i = 0; i < B->nmaps; ++i) {
    size_t most = 0;
    for (int v = 0; v < 2; ++v) {
      int rows = 0, cols = 0, re = 0, ce = 0;
      wf::batch_item_shape(wf::batch_class(B->ny[i], v), &rows, &cols, &re, &ce);
      most = std::max<size_t>(most, std::max<size_t>(B->ny[i] / rows, (B->nx[i] / 2) / cols));
    }
    cap += most;
  }
  B->bd.grid = wf::batch_grid();
  if (B->bd.grid == 0) return WF_EUNSUPPORTED;
  if (cudaStreamCreateWithFlags(&B->pstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return WF_ECUDA;
  }
  wf::BatchDevice& bd = B->bd;
  bd.cap_maps = (size_t)B->nmaps;
  bd.cap_items = cap;
  if (!dalloc(B, &bd.maps, bd.cap_maps) || !dalloc(B, &bd.rows, cap) || !dalloc(B, &bd.cols, cap) ||
      !dalloc(B, &bd.bar, 4) || !dalloc(B, &bd.queue, 2 * (size_t)prm.residual_every) || !dalloc(B, &bd.err, 1))
    return WF_ENOMEM;
  B->plans.assign(B->nmaps, nullptr);
  for (int i = 0; i < B->nmaps; ++i) {
    const int rc = wf_plan_create(&B->plans[i], B->ny[i], B->nx[i], parts, p, B->pstream);
    if (rc != WF_OK) return rc;
  }
  return WF_OK;
}

// wf_solve for every map, the iterations run together (see the top)
int solve_persistent(wf_batch_s* B, const wf_map* maps, const wf_schedule* sched, double tol, wf_stats* stats) {
  const int n = B->nmaps;
  cudaStream_t s = B->pstream;
  if (cudaEventRecord(B->ev_in, B->user) != cudaSuccess || cudaStreamWaitEvent(s, B->ev_in, 0) != cudaSuccess) {
    cudaGetLastError();
    return WF_ECUDA;
  }
  std::vector<wf::SolveJob> J(n);
  std::vector<int> variant(n, 0);
  auto start = [&](int i) {
    const wf_map& m = maps[i];
    J[i] = wf::SolveJob();
    J[i].P = B->plans[i];
    J[i].sched = sched;
    J[i].tol = tol;
    J[i].s_out = m.s_out;
    J[i].st = stats ? &stats[i] : nullptr;
    return wf::job_start(J[i], m.d, m.pixel_var, m.mask, m.C, m.P1f, m.Pst, m.stripe_amp2, nullptr);
  };
  for (int i = 0; i < n; ++i) {
    const int rc = start(i);
    if (rc) return rc;
  }
  // shapes: wf_params.autotune 0 / 2 the first / second, 1 cached per size
  // and device, else timed on the first map of the size
  for (int i = 0; i < n; ++i) {
    const int sz = wf::plan_size(B->plans[i]);
    if (!wf::batch_has_second_shape(sz)) continue;
    const int at = wf::plan_autotune(B->plans[i]);
    if (at != 1) {
      variant[i] = at == 2 ? 1 : 0;
      continue;
    }
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shape.find({sz, B->device});
    if (it == g_shape.end()) {
      double t0 = 0.0, t1 = 0.0;
      int rc = wf::time_batch_variant(B->plans[i], 0, B->bd, s, &t0);
      if (!rc) rc = wf::time_batch_variant(B->plans[i], 1, B->bd, s, &t1);
      if (!rc) rc = start(i);  // the timing sweeps changed the map's state
      if (rc) return rc;
      it = g_shape.emplace(std::make_pair(sz, B->device), (t1 < 0.97 * t0) ? 1 : 0).first;
    }
    variant[i] = it->second;
  }
  auto run = [&](const std::vector<int>& idx, const wf_schedule* sc, double t, std::vector<int>& st_out,
                 std::vector<wf_stats>& s_out) {
    std::vector<wf_plan_t> pl;
    std::vector<int> va;
    for (int i : idx) {
      pl.push_back(B->plans[i]);
      va.push_back(variant[i]);
    }
    return wf::run_plans_persistent(pl, va, sc, t, B->bd, s, st_out, s_out);
  };
  std::vector<int> all(n), st;
  for (int i = 0; i < n; ++i) all[i] = i;
  std::vector<wf_stats> ss;
  int rc = run(all, sched, tol, st, ss);
  if (rc) return rc;
  std::vector<int> active;
  std::vector<int> result(n, WF_OK);
  for (int i = 0; i < n; ++i) {
    bool done = true;
    const int r = wf::job_after_first(J[i], st[i], ss[i], &done);
    if (r) return r;
    if (done) result[i] = J[i].status;
    else active.push_back(i);
  }
  if (!active.empty()) {
    const wf_plan_t P0 = B->plans[active[0]];
    const double ctol = tol * wf::plan_refine_tol_scale(P0);
    auto correction = [&](const std::vector<int>& idx) -> int {
      for (int i : idx) {
        const int r = wf::job_corr_begin(J[i]);
        if (r) return r;
      }
      std::vector<int> cs;
      std::vector<wf_stats> css;
      int r = run(idx, &J[idx[0]].csched, ctol, cs, css);
      if (r) return r;
      for (size_t k = 0; k < idx.size(); ++k)
        if ((r = wf::job_corr_end(J[idx[k]], cs[k], css[k]))) return r;
      return WF_OK;
    };
    for (int r = 0; r < wf::plan_refine(P0); ++r)
      if ((rc = correction(active))) return rc;
    for (int i : active)
      if ((rc = wf::job_refined_residual(J[i]))) return rc;
    // further corrections only for the maps whose refined s fails the stop test
    for (int r = 0; tol > 0 && r < wf::plan_refine_extra(P0); ++r) {
      std::vector<int> failing;
      for (int i : active)
        if (!wf::job_passes(J[i])) failing.push_back(i);
      if (failing.empty()) break;
      if ((rc = correction(failing))) return rc;
      for (int i : failing)
        if ((rc = wf::job_refined_residual(J[i]))) return rc;
    }
    for (int i : active) {
      if ((rc = wf::job_finish(J[i]))) return rc;
      result[i] = J[i].status;
    }
  }
  if (cudaEventRecord(B->ev_out, s) != cudaSuccess || cudaStreamWaitEvent(B->user, B->ev_out, 0) != cudaSuccess) {
    cudaGetLastError();
    return WF_ECUDA;
  }
  int status = WF_OK;
  for (int i = 0; i < n; ++i) {
    if (result[i] != WF_OK && result[i] != WF_ENOCONV && result[i] != WF_ESTALL) return result[i];
    if (result[i] != WF_OK && status == WF_OK) status = result[i];
  }
  return status;
}

}  // namespace

extern "C" {

int wf_batch_create(wf_batch_t* out, int nmaps, const int* ny, const int* nx, unsigned parts,
                    const wf_params* p, int lanes, void* stream) {
  if (!out || !ny || !nx || nmaps < 1 || nmaps > kMaxMaps || lanes < 0 || lanes > kMaxLanes)
    return WF_EINVAL;
  for (int i = 0; i < nmaps; ++i) {
    const int rc = wf::check_plan_args(ny[i], nx[i], parts, p);
    if (rc != WF_OK) return rc;
  }
  if (lanes == 0) {
    const int rc = check_persistent(nmaps, ny, nx, parts, p);
    if (rc != WF_OK) return rc;
  }
  wf_batch_s* B = new wf_batch_s();
  B->nmaps = nmaps;
  B->lanes = std::min(lanes, nmaps);
  B->persistent = (lanes == 0);
  B->ny.assign(ny, ny + nmaps);
  B->nx.assign(nx, nx + nmaps);
  B->user = (cudaStream_t)stream;
  if (cudaGetDevice(&B->device) != cudaSuccess) {
    cudaGetLastError();
    destroy(B);
    return WF_ECUDA;
  }
  if (B->persistent) {
    const int rc = create_persistent(B, parts, p);
    if (rc != WF_OK) {
      destroy(B);
      return rc;
    }
    *out = B;
    return WF_OK;
  }
  // largest first, to the lane with the fewest pixels
  std::vector<int> order(nmaps);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)B->ny[a] * B->nx[a] > (long long)B->ny[b] * B->nx[b];
  });
  B->lane_maps.assign(B->lanes, {});
  std::vector<long long> load(B->lanes, 0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    B->lane_maps[l].push_back(i);
    load[l] += (long long)B->ny[i] * B->nx[i];
  }
  B->lane_stream.assign(B->lanes, nullptr);
  B->lane_done.assign(B->lanes, nullptr);
  B->plans.assign(nmaps, nullptr);
  bool ok = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) == cudaSuccess;
  for (int l = 0; ok && l < B->lanes; ++l) {
    ok = cudaStreamCreateWithFlags(&B->lane_stream[l], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->lane_done[l], cudaEventDisableTiming) == cudaSuccess;
    for (int i : B->lane_maps[l]) {
      if (!ok) break;
      const int rc = wf_plan_create(&B->plans[i], B->ny[i], B->nx[i], parts, p, B->lane_stream[l]);
      if (rc != WF_OK) {
        destroy(B);
        return rc;
      }
    }
  }
  if (!ok) {
    cudaGetLastError();
    destroy(B);
    return WF_ECUDA;
  }
  *out = B;
  return WF_OK;
}

void wf_batch_destroy(wf_batch_t B) {
  if (B) destroy(B);
}

long long wf_batch_launch_count(wf_batch_t B) {
  if (!B) return -1;
  long long n = B->bd.launches;
  for (wf_plan_t p : B->plans) n += wf_launch_count(p);
  return n;
}

int wf_batch_solve(wf_batch_t B, const wf_map* maps, const wf_schedule* sched, double tol, wf_stats* stats) {
  if (!B || !maps || !sched) return WF_EINVAL;
  for (int i = 0; i < B->nmaps; ++i)
    if (!maps[i].d || !maps[i].pixel_var || !maps[i].C || !maps[i].s_out) return WF_EINVAL;
  if (B->persistent) return solve_persistent(B, maps, sched, tol, stats);
  // the lanes start after the caller's work already on its stream
  if (cudaEventRecord(B->ev_in, B->user) != cudaSuccess) {
    cudaGetLastError();
    return WF_ECUDA;
  }
  for (int l = 0; l < B->lanes; ++l)
    if (cudaStreamWaitEvent(B->lane_stream[l], B->ev_in, 0) != cudaSuccess) {
      cudaGetLastError();
      return WF_ECUDA;
    }
  std::vector<int> rc(B->nmaps, WF_OK);
  std::atomic<bool> failed{false};
  auto lane = [&](int l) {
    if (cudaSetDevice(B->device) != cudaSuccess) {
      cudaGetLastError();
      for (int i : B->lane_maps[l]) rc[i] = WF_ECUDA;
      failed = true;
      return;
    }
    for (int i : B->lane_maps[l]) {
      if (failed.load()) {
        rc[i] = kNotRun;  // another map failed: this one is not solved
        continue;
      }
      const wf_map& m = maps[i];
      wf_stats st{};
      rc[i] = wf_solve(B->plans[i], m.d, m.pixel_var, m.mask, m.C, m.P1f, m.Pst, m.stripe_amp2, sched, tol,
                       m.s_out, &st);
      if (stats) stats[i] = st;
      if (rc[i] != WF_OK && rc[i] != WF_ENOCONV && rc[i] != WF_ESTALL) failed = true;
    }
    if (cudaEventRecord(B->lane_done[l], B->lane_stream[l]) != cudaSuccess) cudaGetLastError();
  };
  // every lane on a worker thread: the caller's thread keeps its device
  std::vector<std::thread> th;
  for (int l = 0; l < B->lanes; ++l) th.emplace_back(lane, l);
  for (auto& t : th) t.join();
  // the caller's later work waits for every lane
  for (int l = 0; l < B->lanes; ++l)
    if (cudaStreamWaitEvent(B->user, B->lane_done[l], 0) != cudaSuccess) cudaGetLastError();
  // the first real error (maps skipped after it do not mask it)
  for (int i = 0; i < B->nmaps; ++i)
    if (rc[i] != kNotRun && rc[i] != WF_OK && rc[i] != WF_ENOCONV && rc[i] != WF_ESTALL) return rc[i];
  int status = WF_OK;
  for (int i = 0; i < B->nmaps; ++i) {
    if (rc[i] != WF_OK && rc[i] != WF_ENOCONV && rc[i] != WF_ESTALL) return rc[i];
    if (rc[i] != WF_OK && status == WF_OK) status = rc[i];
  }
  return status;
}

}  // extern "C"
