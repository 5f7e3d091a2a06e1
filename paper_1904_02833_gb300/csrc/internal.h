// Internal structures shared by the solver kernel and the host runtime.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "snakesim.h"

namespace snakesim {

// Layout of one lane group: G lanes per snake, NPL nodes per lane.
constexpr int layout_id(int G, int NPL) { return (G == 8 ? 0 : G == 16 ? 1 : 2) * 4 + (NPL - 1); }
constexpr int layout_lanes(int id) { return 8 << (id / 4); }
constexpr int layout_npl(int id) { return id % 4 + 1; }
constexpr int kNumLayouts = 12;

// Row kinds whose warm-start features are written: in the learned warm start the kinds
// the network predicts (the first 6, 3 or 1 of stretch, yaw, pitch, contact, friction
// x / y), otherwise all six.
__host__ __device__ inline int feature_kinds(int warm, int net_rows) {
  if (warm != SIM_WARM_LEARNED) return 6;
  return net_rows == SIM_NET_ROWS_BILATERAL ? 3 : net_rows == SIM_NET_ROWS_STRETCH ? 1 : 6;
}
// Row slot k of node i (six per node: stretch to i + 1, yaw and pitch bend centred on
// i, contact, friction x / y) of a snake of N nodes whose first nfix nodes are held:
// whether the row exists and is of one of the first nk kinds, i.e. whether its
// warm-start features carry a row kind.
__host__ __device__ inline bool feature_row_exists(int i, int k, int N, int nfix, int contact, int nk) {
  if (k >= nk) return false;
  if (k == 0) return i + 1 <= N - 1;
  if (k <= 2) return i >= 1 && i + 1 <= N - 1;
  return contact != 0 && i >= nfix;
}
// Such rows of the node slots before node i (node by node, kinds in order).
__host__ __device__ inline int feature_rows_before(int i, int N, int nfix, int contact, int nk) {
  const int st = i < N - 1 ? i : N - 1;   // stretch rows of nodes 0 .. min(i, N - 1) - 1
  const int bd = st > 1 ? st - 1 : 0;     // bend pairs of nodes 1 .. min(i, N - 1) - 1
  const int ct = contact != 0 && i > nfix ? i - nfix : 0;
  return st + (nk >= 3 ? 2 * bd : 0) + (nk >= 6 ? 3 * ct : 0);
}

struct SolverArgs {
  float4* pos;            // [nodes] x, y, z, inverse mass
  float4* vel;            // [nodes] vx, vy, vz, 0
  float2* press;          // [links] p_R, p_L
  float* lam;             // [nodes][6]
  const SnakeParams* prm; // [snakes]
  const int* node_off;    // [snakes + 1]
  const int* link_off;    // [snakes + 1]
  float* resid;           // [snakes]
  int* iters;             // [snakes]
  int* status;            // [snakes]
  const int4* items;      // [n_items] (offset into order, snakes in item, layout id, 0)
  const int* order;       // snake indices grouped by layout
  const int* feat_off;    // [snakes] first node of the snake in the feature / lam0 row order
  int n_items;
  int* work;              // work-queue counter of this launch (zeroed before the launch)
  const float* ucmd;      // [links] command override or null
  const float* lam0;      // learned warm start, normalised multipliers [nodes][6] or null
  __nv_bfloat16* feat;    // warm-start features [nodes * 6][32] (split mode)
  int split;              // 0: fused env-steps; 1: one substep boundary per launch
  int sub;                // split mode: substep to finish (-1: none, begin substep 0)
  const long long* step_dev;  // device env-step counter (time = counter * dt)
  long long total_nodes;
  int n_steps;
  double h_d;
  float h;
  int n_sub;
  int K;
  float tol;
  float omega;
  float g[3];
  int contact;
  int warm;
  float beta;
  int latency;            // SIM_LATENCY_*
  int law_every;          // SIM_LATENCY_LAW: substeps per law step
  float k_i, k_d, t_p, p_s;
  int pcr_iters;          // SIM_SOLVER_NEWTON_PCR: PCR iterations per Newton step
  int net_rows;           // SIM_WARM_LEARNED: SIM_NET_ROWS_*
  int net_every;          // SIM_WARM_LEARNED: the network's substeps are multiples of it (>= 1)
  int feat_kinds;         // split mode: row kinds whose features are written (feature_kinds)
  float beta_net;         // SIM_WARM_LEARNED: weight of lambda_prev under the prediction
  int span;               // split mode: substeps the launch finishes (the first one with the
                          // network's start, the others from beta lambda_prev)
};

// Calibration (adjoint) state of a simulator, defined in adjoint.cu.
struct CalibState;
CalibState* calib_new();
void calib_delete(CalibState* c);
SimStatus calib_forward(CalibState& C, const SnakeParams* prm, const int* node_off, const int* link_off,
                        int n_snakes, int n_max, int l_max, const float* theta, int n_steps, int ckpt,
                        long long step0, int n_sub, int K, int contact, double dt, float omega,
                        const float* gvec, float4* pos4, float4* vel4, float2* press2, float* tips,
                        cudaStream_t st, std::string& err);
SimStatus calib_backward(CalibState& C, const SnakeParams* prm, const int* node_off, const int* link_off,
                         const float* tips_bar, float* grad, cudaStream_t st, std::string& err);

// Records the message returned by sim_last_error() on this thread.
void set_last_error(const char* msg);
// Enqueues the warm-start network on `feat` [rows][32] -> out [rows] (no synchronisation).
// sel = SIM_NET_ROWS_*: all rows, the first three of every six (stretch, yaw, pitch of a
// node) or the first of every six (stretch); rows then counts those rows.
SimStatus mlp_forward_launch(MlpHandle* h, const void* feat, long long rows, float* out,
                             cudaStream_t stream, int sel);

}  // namespace snakesim
