// Host runtime and C-ABI of the soft-snake simulator (see include/snakesim.h).
//
// Owns the structure-of-arrays state in HBM (float4 positions with inverse mass,
// float4 velocities, float2 chamber pressures, six multipliers per node), buckets the
// snakes by node count, picks a lane layout per bucket (lanes per snake x nodes per
// lane, optionally by timing them: sim_autotune), rebuilds the work queues on the device
// before every env-step (schedule_kernel) and launches one persistent solver kernel per
// layout (Jacobi, Jacobi with anisotropic friction, or Newton + PCR), directly or through
// a captured CUDA graph; in the learned mode each layout runs its own chain of solver and
// network launches, substep by substep, on its own stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "snakesim.h"
#include "solver.cuh"

using namespace snakesim;

namespace {

thread_local std::string g_err;

SimStatus fail(SimStatus s, const std::string& msg) {
  g_err = msg;
  return s;
}

}  // namespace

void snakesim::set_last_error(const char* msg) { g_err = msg; }

namespace {

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

}  // namespace

// ------------------------------------------------------------------ kernels
// One kernel per lane layout (lanes per snake G x nodes per lane NPL): a launch then
// runs a single code path, and the warps of an SM share their instruction cache.  (One
// kernel for all layouts measured 5-7 issue-stall cycles per instruction waiting for
// instructions, against under one with a kernel per layout.)  The host launches the
// layouts that have work on forked streams, so that the next layout fills the tail of the
// previous one.
// Two blocks of four warps per SM leave the compiler up to 255 registers per thread to
// overlap the independent node slots of a lane's pass (the pass is latency-bound: with
// few warps per scheduler, a warp's own instruction-level parallelism sets its speed).
// Measured against three blocks (168 registers): 16384 snakes 2-5 % faster per env-step,
// 4096 snakes 15-39 % faster.
#ifndef SNAKE_MIN_BLOCKS
#define SNAKE_MIN_BLOCKS 2
#endif
// Persistent: every warp takes the next work item (32/G snakes of one node count) from
// the layout's counter in global memory until none is left.
template <int NPL, int G, bool SPLIT, int VAR>
__global__ void __launch_bounds__(128, SNAKE_MIN_BLOCKS) snake_solver_kernel(SolverArgs A) {
  extern __shared__ float solver_smem[];  // Newton + PCR only (kPcrFloatsPerSlot x 32 NPL per warp)
  const int lane = threadIdx.x & 31;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(A.work, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= A.n_items) break;
    const int4 item = A.items[it];
    const int gi = lane / G;
    const bool ok = gi < item.y;
    const int snake = ok ? A.order[item.x + gi] : 0;
    run_group<NPL, G, SPLIT, VAR>(A, snake, ok, solver_smem);
  }
}

typedef void (*SolverKernel)(SolverArgs);
constexpr int kLayouts = 12;
// [split][solver variant: kVarJacobi, kVarAniso, kVarPcr][layout_id(G, NPL)]
#define SNAKE_KERNELS(S, F)                                                                          \
  {snake_solver_kernel<1, 8, S, F>,  snake_solver_kernel<2, 8, S, F>,  snake_solver_kernel<3, 8, S, F>,  \
   snake_solver_kernel<4, 8, S, F>,  snake_solver_kernel<1, 16, S, F>, snake_solver_kernel<2, 16, S, F>, \
   snake_solver_kernel<3, 16, S, F>, snake_solver_kernel<4, 16, S, F>, snake_solver_kernel<1, 32, S, F>, \
   snake_solver_kernel<2, 32, S, F>, snake_solver_kernel<3, 32, S, F>, snake_solver_kernel<4, 32, S, F>}
const SolverKernel kSolverKernels[2][3][kLayouts] = {
    {SNAKE_KERNELS(false, kVarJacobi), SNAKE_KERNELS(false, kVarAniso), SNAKE_KERNELS(false, kVarPcr)},
    {SNAKE_KERNELS(true, kVarJacobi), SNAKE_KERNELS(true, kVarAniso), SNAKE_KERNELS(true, kVarPcr)}};
// dynamic shared memory of a block of the Newton + PCR kernels
inline size_t pcr_smem_bytes(int lay) { return (size_t)4 * kPcrFloatsPerSlot * 32 * layout_npl(lay) * sizeof(float); }
#undef SNAKE_KERNELS

// ------------------------------------------------------------------ scheduling
// Before every env-step the work queue is rebuilt on the device from the Jacobi updates
// each snake needed in the previous env-step (temporal coherence):
//  * inside a node-count class the snakes are ranked by that count and consecutive
//    snakes of the ranking share a warp (the lane groups of a warp run in lock step until
//    the slowest has converged, so similar snakes waste fewer passes);
//  * inside every layout's queue the items are ordered most expensive first (longest-
//    processing-time order, an item costing about its largest update count), so that
//    the launch does not end on a few long items.
// The physics of a snake does not depend on the warp or the queue position it gets.
struct SchedArgs {
  const int* iters;     // [S] updates of the previous env-step (0: none yet)
  const int* node_off;  // [S + 1]
  const int* cls;       // [S] class of each snake (-1: not scheduled)
  const int* cls_base;  // [C] first slot of the class in `order`
  const int4* items0;   // [n_items] the classes' items (offset, count, layout), class by class
  int* hist;            // [(C + 12) * 256] scratch
  int* key;             // [n_items] scratch
  int* order;           // out: the snakes of class c at [cls_base[c], cls_base[c] + count)
  int4* items;          // out: the queue of layout l at [lay_first[l], lay_first[l + 1])
  int n, n_cls, n_items;
  int lay_first[12];
};

// Predicted cost of a snake: its last update count (its node count before the first step).
__device__ __forceinline__ int sched_cost(const SchedArgs& a, int s) {
  const int v = a.iters[s];
  return min(v > 0 ? v : a.node_off[s + 1] - a.node_off[s], 1 << 26);
}

// 16 bins per octave, counting down so that the expensive come first.
__device__ __forceinline__ int sched_bin(int v) {
  v = max(v, 1);
  const int e = 31 - __clz(v);
  const int m = e >= 4 ? (v >> (e - 4)) & 15 : (v << (4 - e)) & 15;
  return 255 - min(255, 16 * e + m);
}

// In-place exclusive prefix sum of 256 counters by one warp.
__device__ __forceinline__ void warp_scan256(int* c) {
  const int lane = threadIdx.x & 31;
  int v[8], sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = c[lane * 8 + k]; sum += v[k]; }
  int inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  int run = inc - sum;
#pragma unroll
  for (int k = 0; k < 8; ++k) { c[lane * 8 + k] = run; run += v[k]; }
}

// One block: counting sort of the snakes by (class, cost bin), then of the items by
// (layout, cost bin of their first = most expensive snake).
__global__ void __launch_bounds__(1024) schedule_kernel(SchedArgs a) {
  const int t = threadIdx.x, T = blockDim.x, warp = t >> 5, nw = T >> 5;
  int* hi = a.hist + a.n_cls * 256;
  for (int i = t; i < (a.n_cls + 12) * 256; i += T) a.hist[i] = 0;
  __syncthreads();
  for (int s = t; s < a.n; s += T) {
    const int c = a.cls[s];
    if (c >= 0) atomicAdd(&a.hist[c * 256 + sched_bin(sched_cost(a, s))], 1);
  }
  __syncthreads();
  for (int r = warp; r < a.n_cls; r += nw) warp_scan256(a.hist + r * 256);
  __syncthreads();
  for (int s = t; s < a.n; s += T) {
    const int c = a.cls[s];
    if (c >= 0) a.order[a.cls_base[c] + atomicAdd(&a.hist[c * 256 + sched_bin(sched_cost(a, s))], 1)] = s;
  }
  __syncthreads();
  for (int k = t; k < a.n_items; k += T) {
    const int4 it = a.items0[k];
    const int b = sched_bin(sched_cost(a, a.order[it.x]));
    a.key[k] = b;
    atomicAdd(&hi[it.z * 256 + b], 1);
  }
  __syncthreads();
  for (int r = warp; r < 12; r += nw) warp_scan256(hi + r * 256);
  __syncthreads();
  for (int k = t; k < a.n_items; k += T) {
    const int4 it = a.items0[k];
    a.items[a.lay_first[it.z] + atomicAdd(&hi[it.z * 256 + a.key[k]], 1)] = it;
  }
}

// Advances the device env-step counter once all solver launches of a step are done.
__global__ void advance_step_kernel(long long* step, int n) { *step += n; }

__global__ void pack_xyz_kernel(const float4* __restrict__ in, float* __restrict__ out, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) { float4 p = in[i]; out[3 * i] = p.x; out[3 * i + 1] = p.y; out[3 * i + 2] = p.z; }
}

__global__ void unpack_xyz_kernel(const float* __restrict__ in, float4* __restrict__ out, long long n,
                                  const float* __restrict__ inv_mass) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    out[i] = make_float4(in[3 * i], in[3 * i + 1], in[3 * i + 2], inv_mass ? inv_mass[i] : 0.f);
  }
}

// Training rows of the learned warm start (sim_training_rows): one warp per snake, lanes
// over its nodes.  Every existing row of the nk written kinds (feature_row_exists) of
// node i goes to output row out_off[s] + feature_rows_before(i) + (such kinds of node i
// before k): its features
// are copied and its target is (lam_star - beta lam_prev) / (m g h^2), the network's
// output that would turn the warm start beta lam_prev + m g h^2 y into lam_star.
__global__ void training_rows_kernel(const __nv_bfloat16* __restrict__ feat, const int* __restrict__ feat_off,
                                     const int* __restrict__ node_off, const SnakeParams* __restrict__ prm,
                                     const long long* __restrict__ out_off, const float* __restrict__ lam_star,
                                     const float* __restrict__ lam_prev, float beta, float h, int contact,
                                     int nk, int n, __nv_bfloat16* __restrict__ feat_out,
                                     float* __restrict__ target_out) {
  const int s = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= n) return;
  const SnakeParams P = prm[s];
  const int N = P.n_links * P.seg_per_link + 1;
  const float inv = 1.0f / (P.mass * 9.81f * h * h);
  for (int i = lane; i < N; i += 32) {
    long long o = out_off[s] + feature_rows_before(i, N, P.n_fixed, contact, nk);
    const long long g = (long long)node_off[s] + i;
    for (int k = 0; k < 6; ++k) {
      if (!feature_row_exists(i, k, N, P.n_fixed, contact, nk)) continue;
      const uint4* src = reinterpret_cast<const uint4*>(feat + ((long long)(feat_off[s] + i) * 6 + k) * 32);
      uint4* dst = reinterpret_cast<uint4*>(feat_out + o * 32);
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[c] = src[c];
      target_out[o] = (lam_star[g * 6 + k] - beta * lam_prev[g * 6 + k]) * inv;
      ++o;
    }
  }
}

// ------------------------------------------------------------------ handle
struct SimHandle {
  SimConfig cfg;
  int n = 0;
  long long n_nodes = 0, n_links = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<SnakeParams> hprm;
  std::vector<int> node_off, link_off;
  std::vector<float> inv_mass_h;
  // device
  float4 *pos = nullptr, *vel = nullptr;
  float2* press = nullptr;
  float* lam = nullptr;
  SnakeParams* prm = nullptr;
  int *node_off_d = nullptr, *link_off_d = nullptr;
  float* resid = nullptr;
  int *iters = nullptr, *status = nullptr;
  int4* items = nullptr;
  int* order = nullptr;
  int n_items = 0;
  // device scheduling (schedule_kernel): class of each snake, class offsets, scratch
  // feature rows: the snakes of one layout take consecutive rows (network per layout);
  // snake s's rows start at 6 feat_off[s], layout l's nodes are [lay_fnode[l], lay_fnode[l+1])
  int* feat_off_d = nullptr;
  std::vector<int> feat_off;
  long long lay_fnode[kLayouts + 1] = {};
  int4* items0 = nullptr;
  int *sched_cls = nullptr, *sched_base = nullptr, *sched_hist = nullptr, *sched_key = nullptr;
  int n_cls = 0;
  int lay_first[kLayouts + 1] = {};  // items of layout l are [lay_first[l], lay_first[l + 1])
  int lay_grid[kLayouts] = {};
  int lay_launch[kLayouts] = {};      // layouts with work, most work first
  int aniso = 0;                      // some snake has anisotropic friction
  int n_lay = 0;
  int* work = nullptr;                // [kLayouts] work-queue counters
  bool timing = false;                // record an event pair around every solver launch
  struct Timed { int lay; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  cudaStream_t side[kLayouts] = {};
  cudaEvent_t ev_side[kLayouts] = {};
  cudaEvent_t ev_split = nullptr;
  float* ucmd = nullptr;
  bool use_ucmd = false;
  float* inv_mass_d = nullptr;
  float* scratch3 = nullptr;  // [nodes * 6] staging for layout conversions
  float* lam0 = nullptr;            // network output, normalised multipliers [nodes][6]
  __nv_bfloat16* feat = nullptr;   // features [nodes * 6][32]
  MlpHandle* mlp = nullptr;
  CalibState* calib = nullptr;
  int max_nodes = 0, max_links = 0;
  int cur_sub = -1;                // split stepping: substep begun, -1 at a step boundary
  // snapshot
  float4 *snap_pos = nullptr, *snap_vel = nullptr;
  float2* snap_press = nullptr;
  float* snap_lam = nullptr;
  float* snap_resid = nullptr;           // per-snake residual / update count / status
  int *snap_iters = nullptr, *snap_status = nullptr;
  __nv_bfloat16* snap_feat = nullptr;    // features of a begun substep (split stepping)
  long long* train_off = nullptr;        // sim_training_rows: first output row per snake
  std::vector<long long> train_off_h;
  long long snap_step = 0;
  long long* snap_step_dev = nullptr;
  int snap_sub = -1;
  bool snap_valid = false;
  long long step_index = 0;        // host mirror of the device counter
  long long* step_dev = nullptr;   // device env-step counter read by the kernels
  long long launches = 0;
  std::map<int, int> layout;  // node count -> layout id
  int grid = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1;
  long long graph_launches = 0;
  bool graph_dirty = true;
};

namespace {

SimStatus validate_cfg(const SimConfig* c) {
  if (!c) return fail(SIM_EINVAL, "null config");
  if (!(c->dt > 0.0) || c->n_sub < 1 || c->iters < 0 || !(c->tol >= 0.f) || !(c->omega > 0.f) ||
      c->warm < 0 || c->warm > 2 || !(c->beta >= 0.f && c->beta <= 1.f))
    return fail(SIM_EINVAL, "invalid config (dt > 0, n_sub >= 1, iters >= 0, tol >= 0, omega > 0, "
                            "warm in 0..2, beta in [0, 1])");
  if (c->solver != SIM_SOLVER_JACOBI && c->solver != SIM_SOLVER_NEWTON_PCR)
    return fail(SIM_EINVAL, "invalid config: solver must be SIM_SOLVER_JACOBI or SIM_SOLVER_NEWTON_PCR");
  if (c->solver == SIM_SOLVER_NEWTON_PCR && (c->contact != 0 || c->pcr_iters < 1))
    return fail(SIM_EINVAL, "the Newton + PCR solver needs contact = 0 and pcr_iters >= 1");
  if (c->net_rows < SIM_NET_ROWS_ALL || c->net_rows > SIM_NET_ROWS_STRETCH || c->net_every < 0 ||
      !(c->beta_net <= 1.f))
    return fail(SIM_EINVAL, "invalid config: net_rows must be one of SIM_NET_ROWS_*, net_every >= 0, "
                            "beta_net <= 1");
  if (c->latency != SIM_LATENCY_EXP && c->latency != SIM_LATENCY_LAW)
    return fail(SIM_EINVAL, "invalid config: latency must be SIM_LATENCY_EXP or SIM_LATENCY_LAW");
  if (c->latency == SIM_LATENCY_LAW &&
      (!(c->k_inflate > 0.f && c->k_inflate <= 1.f) || !(c->k_deflate > 0.f && c->k_deflate <= 1.f) ||
       !(c->t_p > 0.f) || !(c->p_source > 0.f) || !(c->law_dt >= 0.f)))
    return fail(SIM_EINVAL, "invalid chamber law (k_inflate, k_deflate in (0, 1], t_p > 0, "
                            "p_source > 0, law_dt >= 0)");
  return SIM_OK;
}

int default_layout(int N) {
  for (int G : {8, 16, 32}) {
    if (G * 4 >= N) {
      int npl = (N + G - 1) / G;
      return layout_id(G, std::max(1, npl));
    }
  }
  return -1;
}

// Kernel variant of the handle's configuration and parameters.
int solver_var(const SimHandle* h) {
  if (h->cfg.solver == SIM_SOLVER_NEWTON_PCR) return kVarPcr;
  return h->aniso ? kVarAniso : kVarJacobi;
}

SimStatus build_items(SimHandle* h, const std::map<int, int>* only_bucket = nullptr) {
  // group snakes by node count, pack 32/G snakes per warp item, biggest work first;
  // `only_bucket` restricts the items to the node counts it lists (autotuning)
  std::map<int, std::vector<int>> buckets;
  for (int s = 0; s < h->n; ++s) buckets[h->node_off[s + 1] - h->node_off[s]].push_back(s);
  std::vector<int> order;
  struct It { int off, cnt, lay; float cost; };
  std::vector<It> its;
  std::vector<int> cls(h->n, -1), cls_base;
  for (auto& kv : buckets) {
    if (!h->layout.count(kv.first)) h->layout[kv.first] = default_layout(kv.first);
    if (only_bucket && !only_bucket->count(kv.first)) continue;
    const int lay = h->layout[kv.first];
    if (lay < 0) return fail(SIM_EINVAL, "snake too long for the lane layouts (max 128 nodes)");
    const int G = layout_lanes(lay), per = 32 / G;
    for (int s : kv.second) cls[s] = (int)cls_base.size();
    cls_base.push_back((int)order.size());
    for (size_t b = 0; b < kv.second.size(); b += per) {
      It it;
      it.off = (int)order.size();
      it.cnt = (int)std::min<size_t>(per, kv.second.size() - b);
      it.lay = lay;
      it.cost = (float)kv.first;  // node count: longer snakes take longer
      for (int c = 0; c < it.cnt; ++c) order.push_back(kv.second[b + c]);
      its.push_back(it);
    }
  }
  // items0: class by class (the scheduler's input); the first queue: by layout, longest
  // snakes first inside (before any update counts are known)
  std::vector<int4> items0(its.size());
  for (size_t i = 0; i < its.size(); ++i) items0[i] = make_int4(its[i].off, its[i].cnt, its[i].lay, 0);
  std::stable_sort(its.begin(), its.end(), [](const It& a, const It& b) {
    if (a.lay != b.lay) return a.lay < b.lay;
    return a.cost > b.cost;
  });
  std::vector<int4> hitems(its.size());
  for (size_t i = 0; i < its.size(); ++i) hitems[i] = make_int4(its[i].off, its[i].cnt, its[i].lay, 0);
  for (int4* p : {h->items, h->items0}) if (p) cudaFree(p);
  for (int* p : {h->order, h->sched_cls, h->sched_base, h->sched_hist, h->sched_key}) if (p) cudaFree(p);
  h->items = h->items0 = nullptr;
  h->order = h->sched_cls = h->sched_base = h->sched_hist = h->sched_key = nullptr;
  h->n_items = (int)hitems.size();
  h->n_cls = (int)cls_base.size();
  if (h->n_items > 0) {
    CU(cudaMalloc(&h->items, hitems.size() * sizeof(int4)));
    CU(cudaMalloc(&h->items0, items0.size() * sizeof(int4)));
    CU(cudaMalloc(&h->order, order.size() * sizeof(int)));
    CU(cudaMalloc(&h->sched_cls, h->n * sizeof(int)));
    CU(cudaMalloc(&h->sched_base, cls_base.size() * sizeof(int)));
    CU(cudaMalloc(&h->sched_hist, (cls_base.size() + kLayouts) * 256 * sizeof(int)));
    CU(cudaMalloc(&h->sched_key, hitems.size() * sizeof(int)));
    CU(cudaMemcpy(h->items, hitems.data(), hitems.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->items0, items0.data(), items0.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->sched_cls, cls.data(), h->n * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->sched_base, cls_base.data(), cls_base.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  // feature offsets: layout by layout, snake by snake
  h->feat_off.assign(h->n, 0);
  {
    long long cur = 0;
    for (int l = 0; l < kLayouts; ++l) {
      h->lay_fnode[l] = cur;
      for (auto& kv : buckets) {
        if (h->layout[kv.first] != l || (only_bucket && !only_bucket->count(kv.first))) continue;
        for (int s : kv.second) { h->feat_off[s] = (int)cur; cur += kv.first; }
      }
    }
    h->lay_fnode[kLayouts] = cur;
    // snakes outside the scheduled classes keep their own rows past the end
    for (auto& kv : buckets) {
      if (!(only_bucket && !only_bucket->count(kv.first))) continue;
      for (int s : kv.second) { h->feat_off[s] = (int)cur; cur += kv.first; }
    }
    if (h->feat_off_d) cudaFree(h->feat_off_d);
    h->feat_off_d = nullptr;
    CU(cudaMalloc(&h->feat_off_d, h->n * sizeof(int)));
    CU(cudaMemcpy(h->feat_off_d, h->feat_off.data(), h->n * sizeof(int), cudaMemcpyHostToDevice));
  }
  // per-layout ranges, grids, and launch order (most nodes x nodes per lane first)
  std::vector<double> work(kLayouts, 0.0);
  int cnt[kLayouts] = {};
  for (const It& it : its) { cnt[it.lay] += 1; work[it.lay] += it.cost * layout_npl(it.lay); }
  h->lay_first[0] = 0;
  for (int l = 0; l < kLayouts; ++l) h->lay_first[l + 1] = h->lay_first[l] + cnt[l];
  int dev = 0, sms = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h->n_lay = 0;
  for (int l = 0; l < kLayouts; ++l) {
    h->lay_grid[l] = 0;
    if (cnt[l] == 0) continue;
    int per_sm = 0;
    const int var = solver_var(h);
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kSolverKernels[0][var][l], 128,
                                                     var == kVarPcr ? pcr_smem_bytes(l) : 0));
    const int need = (cnt[l] + 3) / 4;  // four warps per block
    h->lay_grid[l] = std::max(1, std::min(need, std::max(1, per_sm) * sms));
    h->lay_launch[h->n_lay++] = l;
  }
  std::stable_sort(h->lay_launch, h->lay_launch + h->n_lay,
                   [&](int a, int b) { return work[a] > work[b]; });
  h->graph_dirty = true;
  return SIM_OK;
}

SolverArgs make_args(SimHandle* h, int n_steps) {
  SolverArgs A;
  A.pos = h->pos; A.vel = h->vel; A.press = h->press; A.lam = h->lam; A.prm = h->prm;
  A.node_off = h->node_off_d; A.link_off = h->link_off_d;
  A.resid = h->resid; A.iters = h->iters; A.status = h->status;
  A.items = h->items; A.order = h->order; A.n_items = h->n_items;
  A.feat_off = h->feat_off_d;
  A.work = h->work;
  A.ucmd = h->use_ucmd ? h->ucmd : nullptr;
  A.lam0 = (h->cfg.warm == SIM_WARM_LEARNED) ? h->lam0 : nullptr;
  A.feat = h->feat;
  A.split = 0;
  A.sub = -1;
  A.step_dev = h->step_dev;
  A.total_nodes = h->n_nodes;
  A.n_steps = n_steps;
  A.h_d = h->cfg.dt / h->cfg.n_sub;
  A.h = (float)A.h_d;
  A.n_sub = h->cfg.n_sub;
  A.K = h->cfg.iters;
  A.tol = h->cfg.tol;
  A.omega = h->cfg.omega;
  A.g[0] = h->cfg.gravity[0]; A.g[1] = h->cfg.gravity[1]; A.g[2] = h->cfg.gravity[2];
  A.contact = h->cfg.contact;
  A.warm = h->cfg.warm;
  A.beta = h->cfg.beta;
  A.latency = h->cfg.latency;
  A.law_every = std::max(1, (int)std::llround((double)h->cfg.law_dt / A.h_d));
  A.k_i = h->cfg.k_inflate; A.k_d = h->cfg.k_deflate; A.t_p = h->cfg.t_p; A.p_s = h->cfg.p_source;
  A.pcr_iters = h->cfg.pcr_iters;
  A.net_rows = h->cfg.net_rows;
  A.net_every = std::max(1, h->cfg.net_every);
  A.feat_kinds = feature_kinds(h->cfg.warm, h->cfg.net_rows);
  A.beta_net = h->cfg.beta_net < 0.f ? h->cfg.beta : h->cfg.beta_net;
  A.span = 1;
  return A;
}

SimStatus launch_args(SimHandle* h, const SolverArgs& A, cudaStream_t st);
SimStatus launch_layout(SimHandle* h, const SolverArgs& A, int l, cudaStream_t s);
bool forked(const SimHandle* h);
cudaStream_t lay_stream(SimHandle* h, int l, cudaStream_t st);
SimStatus fork_layouts(SimHandle* h, cudaStream_t st);
SimStatus join_layouts(SimHandle* h, cudaStream_t st);
SimStatus launch_net(SimHandle* h, int l, cudaStream_t s);

// Split mode: finish substep `sub` (if >= 0) and begin the next one; with `net`, each
// layout's network launch precedes its solver kernel on the layout's stream.
SimStatus launch_split(SimHandle* h, int sub, cudaStream_t st, bool net) {
  if (h->n_items == 0) return SIM_OK;
  SolverArgs A = make_args(h, 0);
  A.split = 1;
  A.sub = sub;
  SimStatus r = fork_layouts(h, st);
  for (int k = 0; k < h->n_lay && r == SIM_OK; ++k) {
    const int l = h->lay_launch[k];
    cudaStream_t s = lay_stream(h, l, st);
    if (net) r = launch_net(h, l, s);
    if (r == SIM_OK) r = launch_layout(h, A, l, s);
  }
  if (r == SIM_OK) r = join_layouts(h, st);
  return r;
}

// Rebuilds the work queue from the last env-step's update counts.
SimStatus schedule(SimHandle* h, cudaStream_t st) {
  if (h->n_items == 0) return SIM_OK;
  SchedArgs a;
  a.iters = h->iters; a.node_off = h->node_off_d; a.cls = h->sched_cls; a.cls_base = h->sched_base;
  a.items0 = h->items0; a.hist = h->sched_hist; a.key = h->sched_key; a.order = h->order;
  a.items = h->items; a.n = h->n; a.n_cls = h->n_cls; a.n_items = h->n_items;
  for (int l = 0; l < kLayouts; ++l) a.lay_first[l] = h->lay_first[l];
  schedule_kernel<<<1, 1024, 0, st>>>(a);
  CU(cudaGetLastError());
  h->launches += 1;
  return SIM_OK;
}

SimStatus advance(SimHandle* h, int n, cudaStream_t st) {
  advance_step_kernel<<<1, 1, 0, st>>>(h->step_dev, n);
  CU(cudaGetLastError());
  h->launches += 1;
  return SIM_OK;
}

// One env-step in spans of net_every substeps, with the network between solver launches:
// a launch finishes the substep the network has just started and the substeps up to the
// next network substep (those from beta lambda_prev), then begins that one and writes its
// features.  Each layout's chain (solver kernel, network, solver kernel, ...) runs on its
// own stream for the whole env-step: a span of one layout waits only for its own snakes,
// and the other layouts' work fills the tail of its launches.
SimStatus split_step(SimHandle* h, cudaStream_t st) {
  if (h->n_items == 0) return SIM_OK;
  SimStatus r = schedule(h, st);
  if (r == SIM_OK) r = fork_layouts(h, st);
  const bool learned = h->cfg.warm == SIM_WARM_LEARNED;
  const int every = std::max(1, h->cfg.net_every);
  for (int sub = -1; sub < h->cfg.n_sub && r == SIM_OK; sub = sub < 0 ? 0 : sub + every) {
    SolverArgs A = make_args(h, 0);
    A.split = 1;
    A.sub = sub;
    A.span = every;
    for (int k = 0; k < h->n_lay && r == SIM_OK; ++k) {
      const int l = h->lay_launch[k];
      cudaStream_t s = lay_stream(h, l, st);
      if (sub >= 0 && learned) r = launch_net(h, l, s);
      if (r == SIM_OK) r = launch_layout(h, A, l, s);
    }
  }
  if (r == SIM_OK) r = join_layouts(h, st);
  if (r == SIM_OK) r = advance(h, 1, st);
  return r;
}

// Enqueues n_steps env-steps (device counter advanced by the last launch).
SimStatus launch_steps(SimHandle* h, int n_steps, cudaStream_t st) {
  if (n_steps <= 0 || h->n_items == 0) return SIM_OK;
  if (h->cfg.warm == SIM_WARM_LEARNED) {
    for (int k = 0; k < n_steps; ++k) {
      SimStatus r = split_step(h, st);
      if (r != SIM_OK) return r;
    }
    return SIM_OK;
  }
  SimStatus r = schedule(h, st);
  if (r == SIM_OK) r = launch_args(h, make_args(h, n_steps), st);
  if (r == SIM_OK) r = advance(h, n_steps, st);
  return r;
}

// One solver kernel over the items of layout l, on stream s.
SimStatus launch_layout(SimHandle* h, const SolverArgs& A, int l, cudaStream_t s) {
  SolverArgs B = A;
  B.items = h->items + h->lay_first[l];
  B.n_items = h->lay_first[l + 1] - h->lay_first[l];
  B.work = h->work + l;
  CU(cudaMemsetAsync(B.work, 0, sizeof(int), s));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(s, &cap));
  const bool timed = h->timing && cap == cudaStreamCaptureStatusNone;
  SimHandle::Timed tm{l, nullptr, nullptr};
  if (timed) {
    CU(cudaEventCreate(&tm.a));
    CU(cudaEventCreate(&tm.b));
    CU(cudaEventRecord(tm.a, s));
  }
  const int var = solver_var(h);
  kSolverKernels[A.split ? 1 : 0][var][l]<<<h->lay_grid[l], 128, var == kVarPcr ? pcr_smem_bytes(l) : 0, s>>>(B);
  CU(cudaGetLastError());
  if (timed) {
    CU(cudaEventRecord(tm.b, s));
    h->timed.push_back(tm);
  }
  h->launches += 1;
  return SIM_OK;
}

// The layouts' streams: forked from st (or st itself when they run one after another:
// a single layout, or kernel timing on, so that each event pair brackets one kernel).
bool forked(const SimHandle* h) { return h->n_lay > 1 && !h->timing; }
cudaStream_t lay_stream(SimHandle* h, int l, cudaStream_t st) { return forked(h) ? h->side[l] : st; }
SimStatus fork_layouts(SimHandle* h, cudaStream_t st) {
  if (!forked(h)) return SIM_OK;
  CU(cudaEventRecord(h->ev_split, st));
  for (int k = 0; k < h->n_lay; ++k) CU(cudaStreamWaitEvent(h->side[h->lay_launch[k]], h->ev_split, 0));
  return SIM_OK;
}
SimStatus join_layouts(SimHandle* h, cudaStream_t st) {
  if (!forked(h)) return SIM_OK;
  for (int k = 0; k < h->n_lay; ++k) {
    const int l = h->lay_launch[k];
    CU(cudaEventRecord(h->ev_side[l], h->side[l]));
    CU(cudaStreamWaitEvent(st, h->ev_side[l], 0));
  }
  return SIM_OK;
}

// All layouts' kernels of one launch, overlapping on forked streams.
SimStatus launch_args(SimHandle* h, const SolverArgs& A, cudaStream_t st) {
  if (h->n_items == 0) return SIM_OK;
  SimStatus r = fork_layouts(h, st);
  for (int k = 0; k < h->n_lay && r == SIM_OK; ++k) {
    const int l = h->lay_launch[k];
    r = launch_layout(h, A, l, lay_stream(h, l, st));
  }
  if (r == SIM_OK) r = join_layouts(h, st);
  return r;
}

// The network on the feature rows of layout l's snakes (contiguous, see feat_off).
SimStatus launch_net(SimHandle* h, int l, cudaStream_t s) {
  const long long r0 = 6LL * h->lay_fnode[l], r1 = 6LL * h->lay_fnode[l + 1];
  if (r1 <= r0) return SIM_OK;
  const int sel = h->cfg.net_rows;
  const long long rows = sel == SIM_NET_ROWS_BILATERAL ? (r1 - r0) / 2 : (sel == SIM_NET_ROWS_STRETCH ? (r1 - r0) / 6 : r1 - r0);
  SimStatus r = mlp_forward_launch(h->mlp, h->feat + r0 * 32, rows, h->lam0 + r0, s, sel);
  h->launches += 1;
  return r;
}

}  // namespace

// ------------------------------------------------------------------ C-ABI
extern "C" {

const char* sim_last_error(void) { return g_err.c_str(); }

SimStatus sim_create(const SimConfig* cfg, int n_snakes, const SnakeParams* params, void* stream,
                     SimHandle** out) {
  if (!out) return fail(SIM_EINVAL, "null output handle");
  *out = nullptr;
  SimStatus st = validate_cfg(cfg);
  if (st != SIM_OK) return st;
  if (n_snakes < 1 || !params) return fail(SIM_EINVAL, "n_snakes < 1 or null params");
  for (int s = 0; s < n_snakes; ++s) {
    const SnakeParams& p = params[s];
    long long N = (long long)p.n_links * p.seg_per_link + 1;
    if (p.n_links < 1 || p.seg_per_link < 1 || p.n_fixed < 0 || p.n_fixed > N || !(p.L0 > 0.f) ||
        !(p.mass > 0.f) || !(p.alpha_s >= 0.f) || !(p.alpha_b >= 0.f) || !(p.tau_inf > 0.f) ||
        !(p.tau_def > 0.f) || !(p.mu >= 0.f) || !(p.damping >= 0.f) || !(p.mu_side >= 0.f) ||
        (p.mu_side > 0.f && !(p.mu > 0.f)))
      return fail(SIM_EINVAL, "invalid parameters of snake " + std::to_string(s) +
                              " (anisotropic friction needs mu > 0 and mu_side > 0)");
    if (N > 128) return fail(SIM_EINVAL, "snake " + std::to_string(s) + " has more than 128 nodes");
  }
  SimHandle* h = new SimHandle();
  h->cfg = *cfg;
  h->n = n_snakes;
  h->stream = (cudaStream_t)stream;
  h->hprm.assign(params, params + n_snakes);
  for (int s = 0; s < n_snakes; ++s) h->aniso |= params[s].mu_side > 0.f ? 1 : 0;
  h->node_off.resize(n_snakes + 1);
  h->link_off.resize(n_snakes + 1);
  h->node_off[0] = h->link_off[0] = 0;
  for (int s = 0; s < n_snakes; ++s) {
    h->node_off[s + 1] = h->node_off[s] + params[s].n_links * params[s].seg_per_link + 1;
    h->link_off[s + 1] = h->link_off[s] + params[s].n_links;
  }
  h->n_nodes = h->node_off[n_snakes];
  h->n_links = h->link_off[n_snakes];
  for (int s = 0; s < n_snakes; ++s) {
    h->max_nodes = std::max(h->max_nodes, h->node_off[s + 1] - h->node_off[s]);
    h->max_links = std::max(h->max_links, h->link_off[s + 1] - h->link_off[s]);
  }
  auto cleanup = [&](SimStatus s) { sim_destroy(h); return s; };
  // host-side initial pose: straight along yaw0 from (x0, y0, z0), at rest
  std::vector<float4> pos(h->n_nodes), vel(h->n_nodes, make_float4(0.f, 0.f, 0.f, 0.f));
  h->inv_mass_h.resize(h->n_nodes);
  for (int s = 0; s < n_snakes; ++s) {
    const SnakeParams& p = params[s];
    const double c = std::cos((double)p.yaw0), sn = std::sin((double)p.yaw0);
    for (int i = 0; i < h->node_off[s + 1] - h->node_off[s]; ++i) {
      const double d = (double)i * p.L0;
      const float w = (i < p.n_fixed) ? 0.f : 1.0f / p.mass;
      pos[h->node_off[s] + i] = make_float4((float)(p.x0 + d * c), (float)(p.y0 + d * sn), p.z0, w);
      h->inv_mass_h[h->node_off[s] + i] = w;
    }
  }
  cudaError_t e;
#define ALLOC(ptr, bytes)                                                     \
  e = cudaMalloc((void**)&(ptr), (bytes));                                    \
  if (e != cudaSuccess) return cleanup(fail(SIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)));
  ALLOC(h->pos, h->n_nodes * sizeof(float4));
  ALLOC(h->vel, h->n_nodes * sizeof(float4));
  ALLOC(h->press, h->n_links * sizeof(float2));
  ALLOC(h->lam, h->n_nodes * 6 * sizeof(float));
  ALLOC(h->prm, n_snakes * sizeof(SnakeParams));
  ALLOC(h->node_off_d, (n_snakes + 1) * sizeof(int));
  ALLOC(h->link_off_d, (n_snakes + 1) * sizeof(int));
  ALLOC(h->resid, n_snakes * sizeof(float));
  ALLOC(h->iters, n_snakes * sizeof(int));
  ALLOC(h->status, n_snakes * sizeof(int));
  ALLOC(h->ucmd, std::max<long long>(1, h->n_links) * sizeof(float));
  ALLOC(h->inv_mass_d, h->n_nodes * sizeof(float));
  ALLOC(h->scratch3, h->n_nodes * 6 * sizeof(float));
  ALLOC(h->lam0, h->n_nodes * 6 * sizeof(float));
  ALLOC(h->step_dev, sizeof(long long));
  ALLOC(h->work, kLayouts * sizeof(int));
  ALLOC(h->feat, h->n_nodes * 6 * 32 * sizeof(__nv_bfloat16));
#undef ALLOC
#define CUC(call)                                                                         \
  e = (call);                                                                             \
  if (e != cudaSuccess) return cleanup(fail(SIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e)));
  CUC(cudaMemcpy(h->pos, pos.data(), h->n_nodes * sizeof(float4), cudaMemcpyHostToDevice));
  CUC(cudaMemcpy(h->vel, vel.data(), h->n_nodes * sizeof(float4), cudaMemcpyHostToDevice));
  CUC(cudaMemset(h->press, 0, h->n_links * sizeof(float2)));
  CUC(cudaMemset(h->lam, 0, h->n_nodes * 6 * sizeof(float)));
  CUC(cudaMemset(h->feat, 0, h->n_nodes * 6 * 32 * sizeof(__nv_bfloat16)));
  CUC(cudaMemcpy(h->prm, params, n_snakes * sizeof(SnakeParams), cudaMemcpyHostToDevice));
  CUC(cudaMemcpy(h->node_off_d, h->node_off.data(), (n_snakes + 1) * sizeof(int), cudaMemcpyHostToDevice));
  CUC(cudaMemcpy(h->link_off_d, h->link_off.data(), (n_snakes + 1) * sizeof(int), cudaMemcpyHostToDevice));
  CUC(cudaMemset(h->resid, 0, n_snakes * sizeof(float)));
  CUC(cudaMemset(h->iters, 0, n_snakes * sizeof(int)));
  CUC(cudaMemset(h->status, 0, n_snakes * sizeof(int)));
  CUC(cudaMemset(h->step_dev, 0, sizeof(long long)));
  CUC(cudaMemcpy(h->inv_mass_d, h->inv_mass_h.data(), h->n_nodes * sizeof(float), cudaMemcpyHostToDevice));
  CUC(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  CUC(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CUC(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  CUC(cudaEventCreateWithFlags(&h->ev_split, cudaEventDisableTiming));
  for (int l = 0; l < kLayouts; ++l) {
    CUC(cudaStreamCreateWithFlags(&h->side[l], cudaStreamNonBlocking));
    CUC(cudaEventCreateWithFlags(&h->ev_side[l], cudaEventDisableTiming));
  }
#undef CUC
  st = build_items(h);
  if (st != SIM_OK) return cleanup(st);
  *out = h;
  return SIM_OK;
}

SimStatus sim_set_config(SimHandle* h, const SimConfig* cfg) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  SimStatus st = validate_cfg(cfg);
  if (st != SIM_OK) return st;
  const bool regrid = cfg->solver != h->cfg.solver;  // another kernel variant, other occupancy
  h->cfg = *cfg;
  h->graph_dirty = true;
  return regrid ? build_items(h) : SIM_OK;
}

SimStatus sim_set_pressure(SimHandle* h, const float* u, int is_device) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (!u) { h->use_ucmd = false; h->graph_dirty = true; return SIM_OK; }
  CU(cudaMemcpyAsync(h->ucmd, u, h->n_links * sizeof(float),
                     is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  if (!is_device) CU(cudaStreamSynchronize(h->stream));
  if (!h->use_ucmd) h->graph_dirty = true;
  h->use_ucmd = true;
  return SIM_OK;
}

SimStatus sim_step(SimHandle* h, int n_steps) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (n_steps < 0) return fail(SIM_EINVAL, "n_steps < 0");
  if (h->cfg.warm == SIM_WARM_LEARNED && !h->mlp)
    return fail(SIM_EINVAL, "learned warm start requested but no network is attached (sim_set_mlp)");
  if (h->cur_sub >= 0) return fail(SIM_EINVAL, "a split env-step is in progress (sim_split_finish)");
  SimStatus st = launch_steps(h, n_steps, h->stream);
  if (st != SIM_OK) return st;
  h->step_index += n_steps;
  return SIM_OK;
}

SimStatus sim_step_graph(SimHandle* h, int n_steps) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (n_steps < 0) return fail(SIM_EINVAL, "n_steps < 0");
  if (h->cfg.warm == SIM_WARM_LEARNED && !h->mlp)
    return fail(SIM_EINVAL, "learned warm start requested but no network is attached (sim_set_mlp)");
  if (h->cur_sub >= 0) return fail(SIM_EINVAL, "a split env-step is in progress (sim_split_finish)");
  if (n_steps == 0) return SIM_OK;
  // The kernels read the env-step counter from device memory and the graph's last node
  // advances it, so one captured graph per (configuration, layout, n_steps) is replayed
  // unchanged; it is captured on a private stream forked from the handle's stream.
  if (!h->graph || h->graph_dirty || h->graph_steps != n_steps) {
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long launches0 = h->launches;
    SimStatus st = launch_steps(h, n_steps, h->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &g);
    if (st != SIM_OK) { h->launches = launches0; if (g) cudaGraphDestroy(g); return st; }
    if (ce != cudaSuccess) return fail(SIM_ECUDA, std::string("capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) { h->graph = nullptr; return fail(SIM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(ce)); }
    h->graph_steps = n_steps;
    h->graph_dirty = false;
    // kernel launches per replay (counted while capturing)
    h->graph_launches = h->launches - launches0;
    h->launches = launches0;
  }
  CU(cudaEventRecord(h->ev_fork, h->stream));
  CU(cudaStreamWaitEvent(h->cap_stream, h->ev_fork, 0));
  CU(cudaGraphLaunch(h->graph, h->cap_stream));
  CU(cudaEventRecord(h->ev_join, h->cap_stream));
  CU(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  h->launches += h->graph_launches;
  h->step_index += n_steps;
  return SIM_OK;
}

SimStatus sim_get_state(SimHandle* h, float* pos, float* vel, float* press, float* resid,
                        int32_t* iters, int is_device) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  const long long n = h->n_nodes;
  const int blocks = (int)((n + 255) / 256);
  auto kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (pos) {
    float* dst = is_device ? pos : h->scratch3;
    pack_xyz_kernel<<<blocks, 256, 0, h->stream>>>(h->pos, dst, n);
    CU(cudaGetLastError());
    if (!is_device) CU(cudaMemcpyAsync(pos, h->scratch3, n * 3 * sizeof(float), kind, h->stream));
    if (!is_device) CU(cudaStreamSynchronize(h->stream));
  }
  if (vel) {
    float* dst = is_device ? vel : h->scratch3;
    pack_xyz_kernel<<<blocks, 256, 0, h->stream>>>(h->vel, dst, n);
    CU(cudaGetLastError());
    if (!is_device) CU(cudaMemcpyAsync(vel, h->scratch3, n * 3 * sizeof(float), kind, h->stream));
    if (!is_device) CU(cudaStreamSynchronize(h->stream));
  }
  if (press) CU(cudaMemcpyAsync(press, h->press, h->n_links * sizeof(float2), kind, h->stream));
  if (resid) CU(cudaMemcpyAsync(resid, h->resid, h->n * sizeof(float), kind, h->stream));
  if (iters) CU(cudaMemcpyAsync(iters, h->iters, h->n * sizeof(int), kind, h->stream));
  if (!is_device) CU(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

SimStatus sim_set_state(SimHandle* h, const float* pos, const float* vel, const float* press,
                        const float* lam, int is_device) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  const long long n = h->n_nodes;
  const int blocks = (int)((n + 255) / 256);
  auto kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (pos) {
    CU(cudaMemcpyAsync(h->scratch3, pos, n * 3 * sizeof(float), kind, h->stream));
    unpack_xyz_kernel<<<blocks, 256, 0, h->stream>>>(h->scratch3, h->pos, n, h->inv_mass_d);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
  }
  if (vel) {
    CU(cudaMemcpyAsync(h->scratch3, vel, n * 3 * sizeof(float), kind, h->stream));
    unpack_xyz_kernel<<<blocks, 256, 0, h->stream>>>(h->scratch3, h->vel, n, nullptr);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(h->stream));
  }
  if (press) CU(cudaMemcpyAsync(h->press, press, h->n_links * sizeof(float2), kind, h->stream));
  if (lam) CU(cudaMemcpyAsync(h->lam, lam, n * 6 * sizeof(float), kind, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

SimStatus sim_get_lambda(SimHandle* h, float* lam, int is_device) {
  if (!h || !lam) return fail(SIM_EINVAL, "null handle or buffer");
  CU(cudaMemcpyAsync(lam, h->lam, h->n_nodes * 6 * sizeof(float),
                     is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  if (!is_device) CU(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

SimStatus sim_get_info(SimHandle* h, int64_t* n_nodes, int64_t* n_links, int32_t* n_snakes,
                       int64_t* step_index) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (n_nodes) *n_nodes = h->n_nodes;
  if (n_links) *n_links = h->n_links;
  if (n_snakes) *n_snakes = h->n;
  if (step_index) *step_index = h->step_index;
  return SIM_OK;
}

SimStatus sim_set_step_index(SimHandle* h, int64_t step_index) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  h->step_index = step_index;
  long long v = step_index;
  CU(cudaMemcpyAsync(h->step_dev, &v, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return SIM_OK;
}

SimStatus sim_device_state(SimHandle* h, void** pos4, void** vel4, void** press2, void** lam) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (pos4) *pos4 = h->pos;
  if (vel4) *vel4 = h->vel;
  if (press2) *press2 = h->press;
  if (lam) *lam = h->lam;
  return SIM_OK;
}

SimStatus sim_get_status(SimHandle* h, int32_t* status) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  std::vector<int> s(h->n);
  CU(cudaMemcpyAsync(s.data(), h->status, h->n * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  SimStatus worst = SIM_OK;
  for (int i = 0; i < h->n; ++i) {
    if (status) status[i] = s[i];
    if (s[i] == SIM_ENAN) worst = SIM_ENAN;
    else if (s[i] == SIM_NOT_CONVERGED && worst == SIM_OK) worst = SIM_NOT_CONVERGED;
  }
  return worst;
}

SimStatus sim_get_layout(SimHandle* h, int nodes, int32_t* lanes, int32_t* npl) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  auto it = h->layout.find(nodes);
  if (lanes) *lanes = it == h->layout.end() ? 0 : layout_lanes(it->second);
  if (npl) *npl = it == h->layout.end() ? 0 : layout_npl(it->second);
  return SIM_OK;
}

SimStatus sim_set_layout(SimHandle* h, int nodes, int lanes, int npl) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (!(lanes == 8 || lanes == 16 || lanes == 32) || npl < 1 || npl > 4 || lanes * npl < nodes)
    return fail(SIM_EINVAL, "layout needs lanes in {8,16,32}, nodes_per_lane in 1..4, lanes*npl >= nodes");
  h->layout[nodes] = layout_id(lanes, npl);
  return build_items(h);
}

SimStatus sim_autotune(SimHandle* h, int n_steps) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (n_steps < 1) return fail(SIM_EINVAL, "n_steps < 1");
  if (h->cur_sub >= 0) return fail(SIM_EINVAL, "a split env-step is in progress (sim_split_finish)");
  // save the state, time every admissible layout of every bucket alone, restore; every
  // exit goes through `finish`, which frees what was taken, puts the state back and
  // rebuilds the work items of all buckets (with the best layouts, or the old ones on error)
  const long long n = h->n_nodes;
  float4 *p0 = nullptr, *v0 = nullptr;
  float2* pr0 = nullptr;
  float *l0 = nullptr, *r0 = nullptr;
  int *i0 = nullptr, *s0 = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  const std::map<int, int> layout0 = h->layout;
  const long long step_keep = h->step_index;
  SimStatus st = SIM_OK;
  auto ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == SIM_OK)
      st = fail(e == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA, std::string(what) + ": " +
                cudaGetErrorString(e));
    return st == SIM_OK;
  };
  auto copy = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind k) {
    return ok(cudaMemcpyAsync(dst, src, bytes, k, h->stream), "autotune copy");
  };
  auto xfer = [&](bool save) {
    const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
    if (save) {
      return copy(p0, h->pos, n * sizeof(float4), d2d) && copy(v0, h->vel, n * sizeof(float4), d2d) &&
             copy(pr0, h->press, h->n_links * sizeof(float2), d2d) && copy(l0, h->lam, n * 6 * sizeof(float), d2d) &&
             copy(r0, h->resid, h->n * sizeof(float), d2d) && copy(i0, h->iters, h->n * sizeof(int), d2d) &&
             copy(s0, h->status, h->n * sizeof(int), d2d);
    }
    return copy(h->step_dev, &step_keep, sizeof(long long), cudaMemcpyHostToDevice) &&
           copy(h->pos, p0, n * sizeof(float4), d2d) && copy(h->vel, v0, n * sizeof(float4), d2d) &&
           copy(h->press, pr0, h->n_links * sizeof(float2), d2d) && copy(h->lam, l0, n * 6 * sizeof(float), d2d) &&
           copy(h->resid, r0, h->n * sizeof(float), d2d) && copy(h->iters, i0, h->n * sizeof(int), d2d) &&
           copy(h->status, s0, h->n * sizeof(int), d2d);
  };
  std::map<int, int> best = layout0;
  bool saved = false;
  if (ok(cudaMalloc(&p0, n * sizeof(float4)), "cudaMalloc") && ok(cudaMalloc(&v0, n * sizeof(float4)), "cudaMalloc") &&
      ok(cudaMalloc(&pr0, h->n_links * sizeof(float2)), "cudaMalloc") &&
      ok(cudaMalloc(&l0, n * 6 * sizeof(float)), "cudaMalloc") && ok(cudaMalloc(&r0, h->n * sizeof(float)), "cudaMalloc") &&
      ok(cudaMalloc(&i0, h->n * sizeof(int)), "cudaMalloc") && ok(cudaMalloc(&s0, h->n * sizeof(int)), "cudaMalloc") &&
      ok(cudaEventCreate(&a), "cudaEventCreate") && ok(cudaEventCreate(&b), "cudaEventCreate"))
    saved = xfer(true);
  for (auto it = layout0.begin(); st == SIM_OK && it != layout0.end(); ++it) {
    const int N = it->first;
    float best_ms = 1e30f;
    for (int G : {8, 16, 32}) {
      for (int npl = 1; npl <= 4 && st == SIM_OK; ++npl) {
        if (G * npl < N || (npl > 1 && G * (npl - 1) >= N)) continue;  // no empty lanes column
        std::map<int, int> one;
        one[N] = layout_id(G, npl);
        h->layout = layout0;
        h->layout[N] = layout_id(G, npl);
        if ((st = build_items(h, &one)) != SIM_OK) break;
        float ms = 0.f;
        for (int rep = 0; rep < 2 && st == SIM_OK; ++rep) {
          if (!xfer(false) || !ok(cudaEventRecord(a, h->stream), "cudaEventRecord")) break;
          if ((st = launch_steps(h, n_steps, h->stream)) != SIM_OK) break;
          if (!ok(cudaEventRecord(b, h->stream), "cudaEventRecord") || !ok(cudaEventSynchronize(b), "cudaEventSynchronize") ||
              !ok(cudaEventElapsedTime(&ms, a, b), "cudaEventElapsedTime"))
            break;
        }
        if (st == SIM_OK && ms < best_ms) { best_ms = ms; best[N] = layout_id(G, npl); }
      }
    }
  }
  // finish: state back, buffers and events freed, all buckets' items rebuilt
  const SimStatus run = st;
  st = SIM_OK;
  if (saved) xfer(false);
  ok(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
  const SimStatus put_back = st;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  for (void* q : {(void*)p0, (void*)v0, (void*)pr0, (void*)l0, (void*)r0, (void*)i0, (void*)s0})
    if (q) cudaFree(q);
  h->layout = run == SIM_OK ? best : layout0;
  const SimStatus rebuilt = build_items(h);
  if (run != SIM_OK) return run;
  if (put_back != SIM_OK) return put_back;
  return rebuilt;
}

SimStatus sim_set_mlp(SimHandle* h, MlpHandle* m) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  h->mlp = m;
  h->graph_dirty = true;
  return SIM_OK;
}

SimStatus sim_split_begin(SimHandle* h) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (h->cur_sub >= 0) return fail(SIM_EINVAL, "an env-step is already in progress");
  SimStatus st = schedule(h, h->stream);
  if (st == SIM_OK) st = launch_split(h, -1, h->stream, false);
  if (st != SIM_OK) return st;
  h->cur_sub = 0;
  return SIM_OK;
}

SimStatus sim_split_finish(SimHandle* h) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (h->cur_sub < 0) return fail(SIM_EINVAL, "no env-step in progress (sim_split_begin)");
  const bool learned = h->cfg.warm == SIM_WARM_LEARNED;
  if (learned && !h->mlp) return fail(SIM_EINVAL, "learned warm start without a network (sim_set_mlp)");
  const bool net = learned && h->cur_sub % std::max(1, h->cfg.net_every) == 0;
  SimStatus st = launch_split(h, h->cur_sub, h->stream, net);
  if (st != SIM_OK) return st;
  h->cur_sub += 1;
  if (h->cur_sub >= h->cfg.n_sub) {
    st = advance(h, 1, h->stream);
    if (st != SIM_OK) return st;
    h->cur_sub = -1;
    h->step_index += 1;
  }
  return SIM_OK;
}

SimStatus sim_feature_offsets(SimHandle* h, int32_t* first_row) {
  if (!h || !first_row) return fail(SIM_EINVAL, "null handle or output");
  for (int s = 0; s < h->n; ++s) first_row[s] = 6 * h->feat_off[s];
  return SIM_OK;
}

SimStatus sim_features(SimHandle* h, void** feat, int64_t* rows) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (feat) *feat = h->feat;
  if (rows) *rows = h->n_nodes * 6;
  return SIM_OK;
}

SimStatus sim_training_rows(SimHandle* h, const float* lam_star, const float* lam_prev, float beta,
                            void* feat_out, float* target_out, int64_t capacity, int64_t* n_rows) {
  if (!h || !n_rows) return fail(SIM_EINVAL, "null handle or row count");
  if (h->cur_sub < 0) return fail(SIM_EINVAL, "no substep in progress (sim_split_begin)");
  const int contact = h->cfg.contact;
  const int nk = feature_kinds(h->cfg.warm, h->cfg.net_rows);
  h->train_off_h.assign(h->n + 1, 0);
  for (int s = 0; s < h->n; ++s) {
    const SnakeParams& p = h->hprm[s];
    const int N = p.n_links * p.seg_per_link + 1;
    h->train_off_h[s + 1] = h->train_off_h[s] + feature_rows_before(N, N, p.n_fixed, contact, nk);
  }
  const long long total = h->train_off_h[h->n];
  *n_rows = total;
  if (!feat_out && !target_out) return SIM_OK;  // count only
  if (!feat_out || !target_out || !lam_star || !lam_prev)
    return fail(SIM_EINVAL, "null feature, target or multiplier buffer");
  if (capacity < total) return fail(SIM_EINVAL, "output capacity below the row count");
  if (((uintptr_t)feat_out & 15u) != 0) return fail(SIM_EINVAL, "feat_out is not 16-byte aligned");
  if (!(beta >= 0.f && beta <= 1.f)) return fail(SIM_EINVAL, "beta outside [0, 1]");
  if (!h->train_off) CU(cudaMalloc(&h->train_off, (h->n + 1) * sizeof(long long)));
  CU(cudaMemcpyAsync(h->train_off, h->train_off_h.data(), (h->n + 1) * sizeof(long long),
                     cudaMemcpyHostToDevice, h->stream));
  const int threads = 256, blocks = (int)((32LL * h->n + threads - 1) / threads);
  training_rows_kernel<<<blocks, threads, 0, h->stream>>>(
      h->feat, h->feat_off_d, h->node_off_d, h->prm, h->train_off, lam_star, lam_prev, beta,
      (float)(h->cfg.dt / h->cfg.n_sub), contact, nk, h->n, (__nv_bfloat16*)feat_out, target_out);
  CU(cudaGetLastError());
  h->launches += 1;
  return SIM_OK;
}

SimStatus sim_snapshot_save(SimHandle* h) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  const long long n = h->n_nodes;
  if (!h->snap_pos) {
    CU(cudaMalloc(&h->snap_pos, n * sizeof(float4)));
    CU(cudaMalloc(&h->snap_vel, n * sizeof(float4)));
    CU(cudaMalloc(&h->snap_press, h->n_links * sizeof(float2)));
    CU(cudaMalloc(&h->snap_lam, n * 6 * sizeof(float)));
    CU(cudaMalloc(&h->snap_step_dev, sizeof(long long)));
  }
  CU(cudaMemcpyAsync(h->snap_step_dev, h->step_dev, sizeof(long long), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->snap_pos, h->pos, n * sizeof(float4), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->snap_vel, h->vel, n * sizeof(float4), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->snap_press, h->press, h->n_links * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->snap_lam, h->lam, n * 6 * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  // split stepping carries the step's residual and update count from launch to launch,
  // and the next launch of a begun substep reads its features
  if (!h->snap_resid) {
    CU(cudaMalloc(&h->snap_resid, h->n * sizeof(float)));
    CU(cudaMalloc(&h->snap_iters, h->n * sizeof(int)));
    CU(cudaMalloc(&h->snap_status, h->n * sizeof(int)));
  }
  CU(cudaMemcpyAsync(h->snap_resid, h->resid, h->n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->snap_iters, h->iters, h->n * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->snap_status, h->status, h->n * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  if (h->cur_sub >= 0) {
    if (!h->snap_feat) CU(cudaMalloc(&h->snap_feat, n * 6 * 32 * sizeof(__nv_bfloat16)));
    CU(cudaMemcpyAsync(h->snap_feat, h->feat, n * 6 * 32 * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice,
                       h->stream));
  }
  h->snap_step = h->step_index;
  h->snap_sub = h->cur_sub;
  h->snap_valid = true;
  return SIM_OK;
}

SimStatus sim_snapshot_restore(SimHandle* h) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  if (!h->snap_valid) return fail(SIM_EINVAL, "no snapshot saved");
  const long long n = h->n_nodes;
  CU(cudaMemcpyAsync(h->pos, h->snap_pos, n * sizeof(float4), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->vel, h->snap_vel, n * sizeof(float4), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->press, h->snap_press, h->n_links * sizeof(float2), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->lam, h->snap_lam, n * 6 * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->step_dev, h->snap_step_dev, sizeof(long long), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->resid, h->snap_resid, h->n * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->iters, h->snap_iters, h->n * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(h->status, h->snap_status, h->n * sizeof(int), cudaMemcpyDeviceToDevice, h->stream));
  if (h->snap_sub >= 0)
    CU(cudaMemcpyAsync(h->feat, h->snap_feat, n * 6 * 32 * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice,
                       h->stream));
  h->step_index = h->snap_step;
  h->cur_sub = h->snap_sub;
  return SIM_OK;
}

SimStatus sim_calib_forward(SimHandle* h, const float* theta, int n_steps, int ckpt_every, float* tips) {
  if (!h || !theta || !tips) return fail(SIM_EINVAL, "null handle or buffer");
  if (n_steps < 1 || ckpt_every < 1) return fail(SIM_EINVAL, "n_steps and ckpt_every must be >= 1");
  if (h->cur_sub >= 0) return fail(SIM_EINVAL, "a split env-step is in progress (sim_split_finish)");
  if (h->cfg.latency != SIM_LATENCY_EXP)
    return fail(SIM_EINVAL, "calibration differentiates the first-order chamber model only");
  for (const SnakeParams& p : h->hprm)
    if (p.mu_side > 0.f) return fail(SIM_EINVAL, "calibration differentiates isotropic friction only");
  if (!h->calib) h->calib = calib_new();
  std::string err;
  SimStatus st = calib_forward(*h->calib, h->prm, h->node_off_d, h->link_off_d, h->n, h->max_nodes,
                               h->max_links, theta, n_steps, ckpt_every, h->step_index, h->cfg.n_sub,
                               h->cfg.iters, h->cfg.contact, h->cfg.dt, h->cfg.omega, h->cfg.gravity,
                               h->pos, h->vel, h->press, tips, h->stream, err);
  if (st != SIM_OK) return fail(st, err);
  st = advance(h, n_steps, h->stream);
  if (st != SIM_OK) return st;
  h->step_index += n_steps;
  h->launches += 2 + (n_steps + ckpt_every - 1) / ckpt_every;
  return SIM_OK;
}

SimStatus sim_calib_backward(SimHandle* h, const float* tips_bar, float* grad_theta) {
  if (!h || !tips_bar || !grad_theta) return fail(SIM_EINVAL, "null handle or buffer");
  if (!h->calib) return fail(SIM_EINVAL, "no calibration forward pass to differentiate");
  std::string err;
  SimStatus st = calib_backward(*h->calib, h->prm, h->node_off_d, h->link_off_d, tips_bar, grad_theta,
                                h->stream, err);
  if (st != SIM_OK) return fail(st, err);
  return SIM_OK;
}

SimStatus sim_launch_count(SimHandle* h, int64_t* launches) {
  if (!h || !launches) return fail(SIM_EINVAL, "null handle or output");
  *launches = h->launches;
  return SIM_OK;
}

SimStatus sim_kernel_timing(SimHandle* h, int enable) {
  if (!h) return fail(SIM_EINVAL, "null handle");
  h->timing = enable != 0;
  return SIM_OK;
}

SimStatus sim_kernel_times(SimHandle* h, float* ms, int64_t* launches) {
  if (!h || !ms || !launches) return fail(SIM_EINVAL, "null handle or output");
  for (int l = 0; l < kLayouts; ++l) { ms[l] = 0.f; launches[l] = 0; }
  CU(cudaStreamSynchronize(h->stream));
  SimStatus st = SIM_OK;
  for (auto& t : h->timed) {
    float e = 0.f;
    if (st == SIM_OK && cudaEventElapsedTime(&e, t.a, t.b) != cudaSuccess) st = fail(SIM_ECUDA, "event timing");
    ms[t.lay] += e;
    launches[t.lay] += 1;
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  h->timed.clear();
  return st;
}

SimStatus sim_partition(int n_snakes, const SnakeParams* params, int parts, int32_t* first) {
  if (n_snakes < 1 || parts < 1 || !params || !first) return fail(SIM_EINVAL, "n_snakes, parts >= 1 and buffers");
  std::vector<long long> pre(n_snakes + 1, 0);
  for (int s = 0; s < n_snakes; ++s) {
    if (params[s].n_links < 1 || params[s].seg_per_link < 1)
      return fail(SIM_EINVAL, "snake " + std::to_string(s) + " has no links or segments");
    pre[s + 1] = pre[s] + (long long)params[s].n_links * params[s].seg_per_link + 1;
  }
  const long long total = pre[n_snakes];
  first[0] = 0;
  int s = 0;
  for (int p = 1; p < parts; ++p) {
    // nearest boundary to p / parts of the total: |parts pre[s] - p total| smallest
    const long long target = (long long)p * total;
    while (s < n_snakes && (long long)parts * pre[s + 1] <= target) ++s;
    if (s < n_snakes) {
      const long long below = target - (long long)parts * pre[s], above = (long long)parts * pre[s + 1] - target;
      if (above < below) ++s;
    }
    first[p] = std::max(first[p - 1], s);
  }
  first[parts] = n_snakes;
  return SIM_OK;
}

SimStatus sim_destroy(SimHandle* h) {
  if (!h) return SIM_OK;
  cudaStreamSynchronize(h->stream);
  for (auto& t : h->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->calib) calib_delete(h->calib);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_split) cudaEventDestroy(h->ev_split);
  for (int l = 0; l < kLayouts; ++l) {
    if (h->side[l]) cudaStreamDestroy(h->side[l]);
    if (h->ev_side[l]) cudaEventDestroy(h->ev_side[l]);
  }
  void* ptrs[] = {h->pos, h->vel, h->press, h->lam, h->prm, h->node_off_d, h->link_off_d, h->resid,
                  h->iters, h->status, h->items, h->order, h->ucmd, h->inv_mass_d, h->scratch3,
                  h->lam0, h->feat, h->snap_pos, h->snap_vel, h->snap_press, h->snap_lam,
                  h->step_dev, h->snap_step_dev, h->work, h->sched_cls, h->sched_base,
                  h->sched_hist, h->sched_key, h->items0, h->feat_off_d, h->snap_resid,
                  h->snap_iters, h->snap_status, h->snap_feat, h->train_off};
  for (void* p : ptrs) if (p) cudaFree(p);
  delete h;
  return SIM_OK;
}

}  // extern "C"
