// Internal structures shared by the solver kernel and the host runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "snakesim.h"

namespace snakesim {

// Layout of one lane group: G lanes per snake, NPL nodes per lane.
constexpr int layout_id(int G, int NPL) { return (G == 8 ? 0 : G == 16 ? 1 : 2) * 4 + (NPL - 1); }
constexpr int layout_lanes(int id) { return 8 << (id / 4); }
constexpr int layout_npl(int id) { return id % 4 + 1; }
constexpr int kNumLayouts = 12;

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
  int n_items;
  const float* ucmd;      // [links] command override or null
  const float* lam0;      // learned warm start [n_sub][nodes][6] or null
  float* lam_log;         // converged multipliers per substep [n_sub][nodes][6] or null
  long long step_index;
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
};

}  // namespace snakesim
