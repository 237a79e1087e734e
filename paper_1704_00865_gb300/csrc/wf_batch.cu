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
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/wf.h"
#include "wf_internal.h"

struct wf_batch_s {
  int nmaps = 0;
  int lanes = 0;
  int device = 0;
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
  for (cudaEvent_t e : B->lane_done)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : B->lane_stream)
    if (s) cudaStreamDestroy(s);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  delete B;
}

}  // namespace

extern "C" {

int wf_batch_create(wf_batch_t* out, int nmaps, const int* ny, const int* nx, unsigned parts,
                    const wf_params* p, int lanes, void* stream) {
  if (!out || !ny || !nx || nmaps < 1 || nmaps > kMaxMaps || lanes < 1 || lanes > kMaxLanes)
    return WF_EINVAL;
  for (int i = 0; i < nmaps; ++i) {
    const int rc = wf::check_plan_args(ny[i], nx[i], parts, p);
    if (rc != WF_OK) return rc;
  }
  wf_batch_s* B = new wf_batch_s();
  B->nmaps = nmaps;
  B->lanes = std::min(lanes, nmaps);
  B->ny.assign(ny, ny + nmaps);
  B->nx.assign(nx, nx + nmaps);
  B->user = (cudaStream_t)stream;
  if (cudaGetDevice(&B->device) != cudaSuccess) {
    cudaGetLastError();
    destroy(B);
    return WF_ECUDA;
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
  long long n = 0;
  for (wf_plan_t p : B->plans) n += wf_launch_count(p);
  return n;
}

int wf_batch_solve(wf_batch_t B, const wf_map* maps, const wf_schedule* sched, double tol, wf_stats* stats) {
  if (!B || !maps || !sched) return WF_EINVAL;
  for (int i = 0; i < B->nmaps; ++i)
    if (!maps[i].d || !maps[i].pixel_var || !maps[i].C || !maps[i].s_out) return WF_EINVAL;
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
