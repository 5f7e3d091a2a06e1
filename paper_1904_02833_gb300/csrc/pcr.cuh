// Newton + preconditioned conjugate residual (PCR) substep solve on the GPU: the paper's
// own solver structure (Sec. IV-D) over the bilateral rows (stretch, yaw, pitch) of
// contact-free substeps, as an alternative to the Jacobi relaxation.
//
// Each Newton step linearises the rows at x = x_s + d and solves the Schur system of
// Eq. 8, (J M^-1 J^T + alpha~) dlambda = -(c + alpha~ lambda), with `pcr_iters`
// conjugate residual iterations preconditioned by its diagonal (the Jacobi denominators),
// then lambda += dlambda and d += M^-1 J^T dlambda.  Matrix-vector products are counted
// (one per PCR iteration, one per Newton step), like the update count of the Jacobi path.
//
// Layout: the lane group of a snake keeps its multipliers, the Newton increment and the
// CR search directions in registers (rows of its own nodes); the data that neighbouring
// nodes need (segment gradients, the vector being multiplied and M^-1 J^T of it) goes
// through a per-warp shared-memory area indexed by node, each node gathering from the
// rows around it, with __syncwarp() between the phases.
#pragma once

#include "internal.h"

namespace snakesim {

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int off = G / 2; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, G);
  return v;
}

// Shared-memory area of one warp: 32 * NPL node slots; slot = lane * NPL + j, so the
// nodes of a snake (lanes of one group) are consecutive slots.
constexpr int kPcrFloatsPerSlot = 17;
struct PcrSmem {
  float* seg;  // [8][slots] segment i -> i+1: n (3), heading gradient (2), elevation gradient (3)
  float* vin;  // [3][slots] the vector being multiplied (stretch, yaw, pitch rows of node i)
  float* nod;  // [6][slots] x_s and d while linearising; M^-1 J^T v (3) in products
  int slots;
  __device__ float& S(int c, int s) const { return seg[c * slots + s]; }
  __device__ float& V(int c, int s) const { return vin[c * slots + s]; }
  __device__ float& U(int c, int s) const { return nod[c * slots + s]; }
};

__device__ __forceinline__ PcrSmem pcr_smem(float* base, int npl) {
  PcrSmem M;
  M.slots = 32 * npl;
  float* w = base + (threadIdx.x >> 5) * kPcrFloatsPerSlot * M.slots;
  M.seg = w;
  M.vin = w + 8 * M.slots;
  M.nod = w + 11 * M.slots;
  return M;
}

// u_i = w_i (J^T v)_i for the NPL nodes of this lane, gathered from the rows around node
// i (v and the segment gradients read from shared memory; rows that do not exist read 0).
template <int NPL>
__device__ __forceinline__ void pcr_jt(const SnakeK& S, const PcrSmem& M, int q, int base, bool valid,
                                       float (&u)[NPL][3]) {
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = q * NPL + j, s = base + i;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    if (valid && i < S.N && i >= S.nfix) {
      if (i >= 1) {  // stretch(i-1): +n_{i-1}; yaw/pitch(i-1): + segment i-1 gradients
        const float vs = M.V(0, s - 1), vy = M.V(1, s - 1), vp = M.V(2, s - 1);
        a0 += M.S(0, s - 1) * vs + M.S(3, s - 1) * vy + M.S(5, s - 1) * vp;
        a1 += M.S(1, s - 1) * vs + M.S(4, s - 1) * vy + M.S(6, s - 1) * vp;
        a2 += M.S(2, s - 1) * vs + M.S(7, s - 1) * vp;
      }
      {  // rows of node i: stretch -n_i; yaw / pitch -(g_{i-1} + g_i)
        const float vs = M.V(0, s), vy = M.V(1, s), vp = M.V(2, s);
        float gy0 = 0.f, gy1 = 0.f, gp0 = 0.f, gp1 = 0.f, gp2 = 0.f;
        if (i >= 1) { gy0 = M.S(3, s - 1); gy1 = M.S(4, s - 1); gp0 = M.S(5, s - 1); gp1 = M.S(6, s - 1); gp2 = M.S(7, s - 1); }
        gy0 += M.S(3, s); gy1 += M.S(4, s); gp0 += M.S(5, s); gp1 += M.S(6, s); gp2 += M.S(7, s);
        a0 -= M.S(0, s) * vs + gy0 * vy + gp0 * vp;
        a1 -= M.S(1, s) * vs + gy1 * vy + gp1 * vp;
        a2 -= M.S(2, s) * vs + gp2 * vp;
      }
      if (i + 1 <= S.N - 1) {  // yaw/pitch(i+1): + segment i gradients
        const float vy = M.V(1, s + 1), vp = M.V(2, s + 1);
        a0 += M.S(3, s) * vy + M.S(5, s) * vp;
        a1 += M.S(4, s) * vy + M.S(6, s) * vp;
        a2 += M.S(7, s) * vp;
      }
    }
    u[j][0] = S.inv_m * a0; u[j][1] = S.inv_m * a1; u[j][2] = S.inv_m * a2;
  }
}

// y = (J M^-1 J^T + alpha~) v on the rows of this lane's nodes; v[j][r] are this lane's
// entries (0 on rows that do not take part).  Leaves M^-1 J^T v in `u`.
template <int NPL>
__device__ __forceinline__ void pcr_matvec(const SnakeK& S, const PcrSmem& M, int q, int base, bool valid,
                                           const float (&act)[NPL][3], const float (&v)[NPL][3],
                                           float (&y)[NPL][3], float (&u)[NPL][3]) {
#pragma unroll
  for (int j = 0; j < NPL; ++j)
#pragma unroll
    for (int r = 0; r < 3; ++r) M.V(r, base + q * NPL + j) = v[j][r];
  __syncwarp();
  pcr_jt<NPL>(S, M, q, base, valid, u);
#pragma unroll
  for (int j = 0; j < NPL; ++j)
#pragma unroll
    for (int d = 0; d < 3; ++d) M.U(d, base + q * NPL + j) = u[j][d];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = q * NPL + j, s = base + i;
    y[j][0] = y[j][1] = y[j][2] = 0.f;
    if (!(valid && i < S.N)) continue;
    const float ux = u[j][0], uy = u[j][1], uz = u[j][2];
    if (act[j][0] != 0.f) {  // stretch(i): n_i . (u_{i+1} - u_i)
      y[j][0] = M.S(0, s) * (M.U(0, s + 1) - ux) + M.S(1, s) * (M.U(1, s + 1) - uy) +
                M.S(2, s) * (M.U(2, s + 1) - uz) + S.at_s * v[j][0];
    }
    if (act[j][1] != 0.f || act[j][2] != 0.f) {  // yaw / pitch(i): g_{i-1} . (u_{i-1} - u_i) + g_i . (u_{i+1} - u_i)
      const float lx = M.U(0, s - 1) - ux, ly = M.U(1, s - 1) - uy, lz = M.U(2, s - 1) - uz;
      const float rx = M.U(0, s + 1) - ux, ry = M.U(1, s + 1) - uy, rz = M.U(2, s + 1) - uz;
      if (act[j][1] != 0.f)
        y[j][1] = M.S(3, s - 1) * lx + M.S(4, s - 1) * ly + M.S(3, s) * rx + M.S(4, s) * ry + S.at_b * v[j][1];
      if (act[j][2] != 0.f)
        y[j][2] = M.S(5, s - 1) * lx + M.S(6, s - 1) * ly + M.S(7, s - 1) * lz + M.S(5, s) * rx +
                  M.S(6, s) * ry + M.S(7, s) * rz + S.at_b * v[j][2];
    }
  }
  __syncwarp();
}

}  // namespace snakesim
