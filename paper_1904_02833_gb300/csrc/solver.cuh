// Substep solver of the soft-snake chain (sm_103a), register-resident.
//
// One snake is owned by a group of G lanes of a warp (G = 8, 16 or 32); lane q of the
// group owns the NPL consecutive nodes q*NPL .. q*NPL+NPL-1 and keeps their
// substep-start position, displacement within the substep, velocity, the six
// multipliers of the rows they own (stretch to the next node, yaw and pitch bend,
// contact, friction x/y), chamber pressures and rest angles in registers for all
// substeps and env-steps of a launch.
//
// Positions are held as x = x_s + d: x_s (the substep-start position, up to metres from
// the origin) is fixed during the substep and d (a fraction of a millimetre) collects
// the Jacobi corrections.  In FP32 a correction added to x directly is rounded to
// ulp(|x|) ~ 6e-8 m and the late, small corrections are lost, which stalls the
// residual near 1e-4; added to d they keep ~1e-11 m.  Segment vectors are formed as
// (x_s,b - x_s,a) + (d_b - d_a), contact heights as (z_s - r) + d_z, friction slips as d.  Neighbour
// positions and the gradient-times-multiplier contributions that cross a lane boundary
// move by warp shuffles; nothing touches shared or global memory inside the Jacobi loop.
//
// The arithmetic of every step cites the paper (Gasoto et al., arXiv 1904.02833):
//   gait              Eq. 9 (Sec. V-A)
//   chambers          antagonistic pair, Sec. III; first-order latency (exact
//                     exponential relaxation) or the discrete law of Sec. V-A (Eq. 11-12)
//   rest angle        Eq. 3-4 with the inextensible centre layer of Sec. V
//   rows              c + E lambda = 0 (Sec. IV), contact Eq. 7, Coulomb cone (Sec. IV),
//                     optionally anisotropic in the body frame (the wheels of Sec. V)
//   Jacobi relaxation Eq. 8 with its diagonal (Sec. IV-D); or Newton steps with a
//                     preconditioned conjugate residual solve of Eq. 8 (Sec. IV-D,
//                     contact-free substeps; pcr.cuh)
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include <cuda_bf16.h>

#include "internal.h"

namespace snakesim {

constexpr unsigned kFull = 0xffffffffu;

// atan(t) on [-1, 1]: odd polynomial t P(t^2) of degree 8 in t^2, a near-minimax fit
// (Lawson's iteratively reweighted least squares on Chebyshev nodes, tests/fit_atan.py
// prints these float32 coefficients) made for this library; its FP32 evaluation stays
// within ~1.1e-7 of atan (tests/test_fast_atan.py).  Beyond |t| = 1,
// atan(t) = sign(t) pi/2 - atan(1/t).
__device__ __forceinline__ float atan_unit(float t) {
  const float s = t * t;
  float p = 2.456725342e-03f;
  p = fmaf(p, s, -1.440136135e-02f);
  p = fmaf(p, s, 3.978123143e-02f);
  p = fmaf(p, s, -7.234857976e-02f);
  p = fmaf(p, s, 1.049894616e-01f);
  p = fmaf(p, s, -1.416122913e-01f);
  p = fmaf(p, s, 1.998590678e-01f);
  p = fmaf(p, s, -3.333259821e-01f);
  p = fmaf(p, s, 9.999998808e-01f);
  return t * p;
}
__device__ __forceinline__ float atan_any(float t) {
  const float a = fabsf(t);
  const bool big = a > 1.f;
  const float p = atan_unit(big ? __frcp_rn(a) : a);
  return copysignf(big ? 1.57079632679489662f - p : p, t);
}
// atan2(y, x) for the bend angles from the same polynomial, without branches: atan(y / x),
// shifted by +-pi for x < 0, +-pi/2 (0 for y = 0) on the axis x = 0.  (The library atan2f
// would add a large body of code to every solver kernel for the rare angles beyond 90
// degrees.)
__device__ __forceinline__ float atan2_bend(float y, float x) {
  float r = atan_any(__fdividef(y, x));
  r = (x < 0.f) ? r + copysignf(3.14159265358979323846f, y) : r;
  const float axis = (y == 0.f) ? 0.f : copysignf(1.57079632679489662f, y);
  return (x == 0.f) ? axis : r;
}

struct Seg {  // derived quantities of the segment from node i to node i+1
  float ex, ey, ez;   // edge vector
  float len;          // |e|
  float nx, ny, nz;   // e / |e|
  float gyx, gyy;     // L0 d(heading)/de = L0 (-e_y, e_x) / |e_h|^2
  float gpx, gpy, gpz;// L0 d(elevation)/de = L0 (-e_z e_x, -e_z e_y, |e_h|^2) / (|e|^2 |e_h|)
  float beta;         // elevation atan2(e_z, |e_h|) = asin(e_z / |e|)
};

__device__ __forceinline__ Seg make_seg(float ex, float ey, float ez, float L0) {
  Seg s;
  s.ex = ex; s.ey = ey; s.ez = ez;
  const float h2 = s.ex * s.ex + s.ey * s.ey;
  const float l2 = h2 + s.ez * s.ez;
  const float il = rsqrtf(l2);
  s.len = l2 * il;
  s.nx = s.ex * il; s.ny = s.ey * il; s.nz = s.ez * il;
  const float ih = rsqrtf(h2);
  const float ih2 = ih * ih;
  s.gyx = -L0 * s.ey * ih2;
  s.gyy = L0 * s.ex * ih2;
  const float f = L0 * il * il * ih;
  s.gpx = -s.ez * s.ex * f;
  s.gpy = -s.ez * s.ey * f;
  s.gpz = h2 * f;
  s.beta = atan_any(s.ez * ih);  // atan2(e_z, |e_h|), |e_h| > 0
  return s;
}

template <int G>
__device__ __forceinline__ float group_max(float r) {
#pragma unroll
  for (int off = G / 2; off >= 1; off >>= 1) r = fmaxf(r, __shfl_xor_sync(kFull, r, off, G));
  return r;
}

// Per-group constants of one snake.
struct SnakeK {
  int N, seg, nfix, L, nb, lb, fb;  // fb: first node of the snake in the feature row order
  float L0, inv_L0, inv_m, mass, at_s, at_b, mu, radius, gain, e_inf, e_def, damp_over_h;
  float mu_side, inv_mu, inv_mu_side;  // mu_side > 0: anisotropic friction (body frame)
  float om_m;                          // omega m: relaxed contact / friction update per unit slip
};

// Friction pair (px, py) limited to the Coulomb set of normal multiplier ln: the disc
// |p| <= mu ln, or with anisotropic friction (the wheels and scales of Sec. V) the ellipse
// (p_t / mu)^2 + (p_s / mu_side)^2 <= ln^2 in the body frame (t = (bx, by) along the chain,
// s = z x t), projected radially in the coordinates scaled by the two coefficients.
template <bool ANISO>
__device__ __forceinline__ void friction_limit(const SnakeK& S, float bx, float by, float ln, float& px,
                                               float& py) {
  if (ANISO && S.mu_side > 0.f) {
    float a = px * bx + py * by, b = py * bx - px * by;
    const float u = a * S.inv_mu, v = b * S.inv_mu_side;
    const float r2 = u * u + v * v;
    const float sc = (r2 > ln * ln) ? (ln > 0.f ? ln * rsqrtf(r2) : 0.f) : 1.f;
    a *= sc; b *= sc;
    px = a * bx - b * by;
    py = a * by + b * bx;
  } else {
    // scale 1 inside the disc, rad / |p| outside, 0 for an empty disc; no branches
    const float rad = S.mu * ln;
    const float n2 = px * px + py * py;
    const float sc = (n2 > rad * rad) ? (rad > 0.f ? rad * rsqrtf(n2) : 0.f) : 1.f;
    px *= sc; py *= sc;
  }
}

}  // namespace snakesim

#include "pcr.cuh"  // Newton + PCR building blocks (use SnakeK)

namespace snakesim {

// One pass over the rows at the current positions and multipliers.
//   WARM = false: Jacobi pass.  Evaluates every row at (x^k, lambda^k), returns the
//     group's normalised residual, and (unless `stop` comes back true) replaces lambda by
//     its relaxed update and moves every free node by w_i sum_j grad_i c_j d_j.
//   WARM = true: warm-start pass.  Uses d_j = lambda_j (zeroing rows that do not exist
//     or touch no free node) and applies it, so that M (x - x~) = J^T lambda.
// `stop` returns the group's stop decision (residual <= tol or cap reached).
// The pass has no branches on row existence: every row of every node slot is evaluated
// (on a straight dummy segment where the segment does not exist) and a row that does not
// exist contributes d = 0 and residual 0, so that the lane's node slots form independent
// instruction streams the scheduler can interleave.
template <int NPL, int G, bool WARM, bool ANISO>
__device__ __forceinline__ float row_pass(const SnakeK& S, const SolverArgs& A, int q,
                                          bool live, int kiter, const float (&xs)[NPL][3],
                                          float (&dx)[NPL][3], const float (&xsl)[3],
                                          const float (&xsr)[3], float (&lam)[NPL][6],
                                          const float (&th)[NPL], bool& stop) {
  const float L0 = S.L0;
  // neighbour displacements across the lane boundary
  float dxl[3], dxr[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dxl[d] = __shfl_up_sync(kFull, dx[NPL - 1][d], 1, G);
    dxr[d] = __shfl_down_sync(kFull, dx[0][d], 1, G);
  }
  const int i0 = q * NPL;
  // segment i (from node i to node i + 1) from its two end nodes; a straight dummy where
  // the segment does not exist
  auto seg = [&](int u) {
    const int i = i0 + u - 1;
    const bool on = live && i >= 0 && i + 1 <= S.N - 1;
    const float* ax = (u == 0) ? xsl : xs[u > 0 ? u - 1 : 0];
    const float* ad = (u == 0) ? dxl : dx[u > 0 ? u - 1 : 0];
    const float* bx = (u == NPL) ? xsr : xs[u < NPL ? u : 0];
    const float* bd = (u == NPL) ? dxr : dx[u < NPL ? u : 0];
    const float ex = (bx[0] - ax[0]) + (bd[0] - ad[0]);
    const float ey = (bx[1] - ax[1]) + (bd[1] - ad[1]);
    const float ez = (bx[2] - ax[2]) + (bd[2] - ad[2]);
    return make_seg(on ? ex : 1.f, on ? ey : 0.f, on ? ez : 0.f, L0);
  };
  float acc[NPL][3];
  float dl[NPL][6];
  float accL[3] = {0.f, 0.f, 0.f}, accR[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < NPL; ++j) acc[j][0] = acc[j][1] = acc[j][2] = 0.f;
  float r = 0.f, q2 = 0.f;
  Seg sp = seg(0);  // segment i0 - 1
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = i0 + j;
    const Seg sc = seg(j + 1);  // segment i
    const bool act = live && i < S.N;
    const float wi = (i < S.nfix) ? 0.f : S.inv_m;
    const float wl = (i - 1 < S.nfix) ? 0.f : S.inv_m;
    const float wr = (i + 1 < S.nfix) ? 0.f : S.inv_m;
    float* tl = (j > 0) ? acc[j - 1] : accL;          // node i-1
    float* tr = (j + 1 < NPL) ? acc[j + 1] : accR;    // node i+1
    // ---- stretch (i, i+1): c = |e| - L0 (Eq. 3 with a constant rest length)
    {
      const float c = sc.len - L0;
      const float wg = wi + wr;
      const bool on = act && i + 1 <= S.N - 1 && wg > 0.f;
      float d;
      if (WARM) d = lam[j][0];
      else {
        const float l = lam[j][0];
        r = fmaxf(r, on ? fabsf(c + S.at_s * l) : 0.f);
        d = __fdividef(A.omega * (-c - S.at_s * l), wg + S.at_s);
      }
      d = on ? d : 0.f;
      dl[j][0] = d;
      acc[j][0] -= sc.nx * d; acc[j][1] -= sc.ny * d; acc[j][2] -= sc.nz * d;
      tr[0] += sc.nx * d; tr[1] += sc.ny * d; tr[2] += sc.nz * d;
    }
    // ---- yaw and pitch bend centred on node i (rows in length units: L0 x angle)
    const bool bend = act && i >= 1 && i <= S.N - 2;
    // yaw: L0 (atan2(z . (e1 x e2), e1_h . e2_h) - theta_rest)
    {
      const float cz = sp.ex * sc.ey - sp.ey * sc.ex;
      const float dh = sp.ex * sc.ex + sp.ey * sc.ey;
      const float c = L0 * (atan2_bend(cz, dh) - th[j]);
      const float g0x = sp.gyx, g0y = sp.gyy;                     // node i-1
      const float g1x = -sp.gyx - sc.gyx, g1y = -sp.gyy - sc.gyy; // node i
      const float g2x = sc.gyx, g2y = sc.gyy;                     // node i+1
      const float wg = wl * (g0x * g0x + g0y * g0y) + wi * (g1x * g1x + g1y * g1y) +
                       wr * (g2x * g2x + g2y * g2y);
      const bool on = bend && wg > 0.f;
      float d;
      if (WARM) d = lam[j][1];
      else {
        const float l = lam[j][1];
        r = fmaxf(r, on ? fabsf(c + S.at_b * l) : 0.f);
        d = __fdividef(A.omega * (-c - S.at_b * l), wg + S.at_b);
      }
      d = on ? d : 0.f;
      dl[j][1] = d;
      tl[0] += g0x * d; tl[1] += g0y * d;
      acc[j][0] += g1x * d; acc[j][1] += g1y * d;
      tr[0] += g2x * d; tr[1] += g2y * d;
    }
    // pitch: L0 (elevation(e2) - elevation(e1))
    {
      const float c = L0 * (sc.beta - sp.beta);
      const float g0x = sp.gpx, g0y = sp.gpy, g0z = sp.gpz;
      const float g1x = -sp.gpx - sc.gpx, g1y = -sp.gpy - sc.gpy, g1z = -sp.gpz - sc.gpz;
      const float g2x = sc.gpx, g2y = sc.gpy, g2z = sc.gpz;
      const float wg = wl * (g0x * g0x + g0y * g0y + g0z * g0z) +
                       wi * (g1x * g1x + g1y * g1y + g1z * g1z) +
                       wr * (g2x * g2x + g2y * g2y + g2z * g2z);
      const bool on = bend && wg > 0.f;
      float d;
      if (WARM) d = lam[j][2];
      else {
        const float l = lam[j][2];
        r = fmaxf(r, on ? fabsf(c + S.at_b * l) : 0.f);
        d = __fdividef(A.omega * (-c - S.at_b * l), wg + S.at_b);
      }
      d = on ? d : 0.f;
      dl[j][2] = d;
      tl[0] += g0x * d; tl[1] += g0y * d; tl[2] += g0z * d;
      acc[j][0] += g1x * d; acc[j][1] += g1y * d; acc[j][2] += g1z * d;
      tr[0] += g2x * d; tr[1] += g2y * d; tr[2] += g2z * d;
    }
    sp = sc;
  }
  // ---- ground contact (Eq. 7, z - r >= 0) and Coulomb friction pair of every node slot.
  // Their residual terms decide nothing in a pass where every group's bilateral terms
  // already exceed the tolerance (the group cannot stop) and the cap is not reached, so
  // they are evaluated only when some group's could decide it (warp-uniform choice
  // between two compiled forms of the loop); the updates are the same either way.
  auto contact_rows = [&](auto with_residual) {
    constexpr bool RES = decltype(with_residual)::value;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = i0 + j;
      const bool act = live && i < S.N;
      const float wi = (i < S.nfix) ? 0.f : S.inv_m;
      const bool on = act && A.contact && wi > 0.f;
      const float ln = lam[j][3];
      const float cn = (xs[j][2] - S.radius) + dx[j][2];
      const float ux = dx[j][0], uy = dx[j][1];
      float dn, fx, fy;
      if (WARM) { dn = ln; fx = lam[j][4]; fy = lam[j][5]; }
      else {
        // body tangent at the substep start (anisotropic friction only)
        float bx = 1.f, by = 0.f;
        if (ANISO && S.mu_side > 0.f) {
          float ax0 = xs[j][0], ay0 = xs[j][1], bx0 = xs[j][0], by0 = xs[j][1];
          if (i >= 1) { ax0 = (j > 0) ? xs[j - 1][0] : xsl[0]; ay0 = (j > 0) ? xs[j - 1][1] : xsl[1]; }
          if (i + 1 <= S.N - 1) {
            bx0 = (j + 1 < NPL) ? xs[j + 1][0] : xsr[0];
            by0 = (j + 1 < NPL) ? xs[j + 1][1] : xsr[1];
          }
          const float ex = bx0 - ax0, ey = by0 - ay0, en2 = ex * ex + ey * ey;
          if (en2 > 0.f) { const float ie = rsqrtf(en2); bx = ex * ie; by = ey * ie; }
        }
        if constexpr (RES) {
          // residuals: Fischer-Burmeister on (c_n, w lambda_n); natural map of the cone
          const float b = wi * ln;
          r = fmaxf(r, on ? fabsf(cn + b - sqrtf(cn * cn + b * b)) : 0.f);
          const float ax = wi * lam[j][4], ay = wi * lam[j][5];
          float px = ax - ux, py = ay - uy;
          friction_limit<ANISO>(S, bx, by, wi * ln, px, py);
          // squared friction residual; one square root per pass for the whole lane
          q2 = fmaxf(q2, on ? (ax - px) * (ax - px) + (ay - py) * (ay - py) : 0.f);
        }
        // contact: lambda_n <- max(0, lambda_n + omega (-c_n / w))
        const float nl = fmaxf(0.f, ln - S.om_m * cn);
        dn = nl - ln;
        // friction: relaxed update limited to the Coulomb set of the current iterate's
        // lambda_n
        float tx = lam[j][4] - S.om_m * ux;
        float ty = lam[j][5] - S.om_m * uy;
        friction_limit<ANISO>(S, bx, by, ln, tx, ty);
        fx = tx - lam[j][4]; fy = ty - lam[j][5];
      }
      dn = on ? dn : 0.f; fx = on ? fx : 0.f; fy = on ? fy : 0.f;
      dl[j][3] = dn; dl[j][4] = fx; dl[j][5] = fy;
      acc[j][2] += dn;
      acc[j][0] += fx;
      acc[j][1] += fy;
    }
  };
  bool cf_residual = true;
  if (!WARM) {
    // a group could stop only if none of its lanes has a bilateral term over the
    // tolerance (a non-finite term counts as not over, so that it reaches the residual)
    const float rb = r * S.inv_L0;
    const unsigned ln_ = threadIdx.x & 31u;
    const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (ln_ & ~(unsigned)(G - 1)));
    const unsigned over_b = __ballot_sync(kFull, rb > A.tol);
    cf_residual = __any_sync(kFull, live && (over_b & gm) == 0u) || kiter >= A.K;
  }
  if (cf_residual) contact_rows(std::true_type{});
  else contact_rows(std::false_type{});
  if (!WARM) {
    // every term is a length: one scaling by 1 / L0 (monotone, so the max is the same)
    r = fmaxf(r, sqrtf(q2)) * S.inv_L0;
    if (!(r <= 3.0e38f)) r = INFINITY;  // NaN -> inf so that the max keeps it
    // one ballot decides every group's stop; the group's max residual is reduced only in
    // the (rare) passes where some live group stops, to be recorded
    const unsigned lane = threadIdx.x & 31u;
    const unsigned over = __ballot_sync(kFull, !(r <= A.tol));
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
    stop = ((over & gmask) == 0u) || (kiter >= A.K);
    if (__any_sync(kFull, stop && live)) r = group_max<G>(r);
  } else {
    stop = false;
  }
  // contributions that cross lane boundaries
  float fromR[3], fromL[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    fromR[d] = __shfl_down_sync(kFull, accL[d], 1, G);  // right lane's rows -> my last node
    fromL[d] = __shfl_up_sync(kFull, accR[d], 1, G);    // left lane's rows -> my first node
  }
  // update, by selects: a node slot beyond the snake or a group that stops keeps its state
  const bool upd = live && !stop;
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = i0 + j;
    float ax = acc[j][0], ay = acc[j][1], az = acc[j][2];
    if (j == 0 && q > 0) { ax += fromL[0]; ay += fromL[1]; az += fromL[2]; }
    if (j == NPL - 1 && q < G - 1) { ax += fromR[0]; ay += fromR[1]; az += fromR[2]; }
    const bool on = upd && i < S.N;
    const float wi = (i < S.nfix) ? 0.f : S.inv_m;
    dx[j][0] = on ? dx[j][0] + wi * ax : dx[j][0];
    dx[j][1] = on ? dx[j][1] + wi * ay : dx[j][1];
    dx[j][2] = on ? dx[j][2] + wi * az : dx[j][2];
#pragma unroll
    for (int k = 0; k < 6; ++k) lam[j][k] = on ? (WARM ? dl[j][k] : lam[j][k] + dl[j][k]) : lam[j][k];
  }
  return r;
}

// Writes the 24 warm-start features (padded to 32, bf16) of the six rows each node owns,
// at the predicted positions of the substep start.  Row frame: horizontal unit tangent
// t (stretch: its own segment; bend: the incoming segment; contact: the outgoing one;
// friction x / y: world x / y), b = z x t, z.  Features: one-hot row kind (6); height of
// the row's first node above its contact height / L0 (1); positions of the row's second
// and third node relative to the first, in the frame, / L0 (6); velocities of the up to
// three nodes in the frame, x h / L0 (9); rest angle of a yaw row (1); the row's
// multiplier from the previous substep / (m g h^2) (1).  Rows that do not exist are zero;
// only the first A.feat_kinds kinds are written (the kinds the network predicts).
template <int NPL, int G>
__device__ __forceinline__ void write_features(const SnakeK& S, const SolverArgs& A, int q, bool valid,
                                               const float (&xs)[NPL][3], const float (&dx)[NPL][3],
                                               const float (&v)[NPL][3], const float (&lam)[NPL][6],
                                               const float (&th)[NPL]) {
  float nl[9], nr[9];  // left / right neighbour: xs, dx, v
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    nl[d] = __shfl_up_sync(kFull, xs[NPL - 1][d], 1, G);
    nl[3 + d] = __shfl_up_sync(kFull, dx[NPL - 1][d], 1, G);
    nl[6 + d] = __shfl_up_sync(kFull, v[NPL - 1][d], 1, G);
    nr[d] = __shfl_down_sync(kFull, xs[0][d], 1, G);
    nr[3 + d] = __shfl_down_sync(kFull, dx[0][d], 1, G);
    nr[6 + d] = __shfl_down_sync(kFull, v[0][d], 1, G);
  }
  if (!valid) return;
  const float lsc = 1.0f / (S.mass * 9.81f * A.h * A.h);
  const float hl = A.h * S.inv_L0;
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = q * NPL + j;
    if (i >= S.N) continue;
    // nodes i-1, i, i+1: substep-start position, displacement, velocity
    float X[3][3], D[3][3], V[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      X[1][d] = xs[j][d]; D[1][d] = dx[j][d]; V[1][d] = v[j][d];
      if (j > 0) { X[0][d] = xs[j - 1][d]; D[0][d] = dx[j - 1][d]; V[0][d] = v[j - 1][d]; }
      else { X[0][d] = nl[d]; D[0][d] = nl[3 + d]; V[0][d] = nl[6 + d]; }
      if (j + 1 < NPL) { X[2][d] = xs[j + 1][d]; D[2][d] = dx[j + 1][d]; V[2][d] = v[j + 1][d]; }
      else { X[2][d] = nr[d]; D[2][d] = nr[3 + d]; V[2][d] = nr[6 + d]; }
    }
    auto rel = [&](int b, int a, int d) { return (X[b][d] - X[a][d]) + (D[b][d] - D[a][d]); };
    auto dirh = [&](int b, int a, float& tx, float& ty) {
      const float ex = rel(b, a, 0), ey = rel(b, a, 1);
      const float n2 = ex * ex + ey * ey;
      if (n2 > 0.f) { const float in = rsqrtf(n2); tx = ex * in; ty = ey * in; }
      else { tx = 1.f; ty = 0.f; }
    };
    const bool has_next = i + 1 <= S.N - 1;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (k >= A.feat_kinds) break;  // kinds the network does not predict are not written
      float f[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) f[c] = 0.f;
      if (feature_row_exists(i, k, S.N, S.nfix, A.contact, 6)) {
        f[k] = 1.f;
        int na, nb = -1, nc = -1;  // local node indices 0..2 (i-1, i, i+1)
        float tx, ty;
        if (k == 0) { na = 1; nb = 2; dirh(2, 1, tx, ty); }
        else if (k <= 2) { na = 0; nb = 1; nc = 2; dirh(1, 0, tx, ty); }
        else {
          na = 1;
          if (k == 3) { if (has_next) dirh(2, 1, tx, ty); else dirh(1, 0, tx, ty); }
          else if (k == 4) { tx = 1.f; ty = 0.f; }
          else { tx = 0.f; ty = 1.f; }
        }
        f[6] = ((X[na][2] - S.radius) + D[na][2]) * S.inv_L0;
        if (nb >= 0) {
          const float ux = rel(nb, na, 0), uy = rel(nb, na, 1), uz = rel(nb, na, 2);
          f[7] = (ux * tx + uy * ty) * S.inv_L0;
          f[8] = (-ux * ty + uy * tx) * S.inv_L0;
          f[9] = uz * S.inv_L0;
        }
        if (nc >= 0) {
          const float ux = rel(nc, na, 0), uy = rel(nc, na, 1), uz = rel(nc, na, 2);
          f[10] = (ux * tx + uy * ty) * S.inv_L0;
          f[11] = (-ux * ty + uy * tx) * S.inv_L0;
          f[12] = uz * S.inv_L0;
        }
        const int nodes[3] = {na, nb, nc};
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          if (nodes[u] < 0) continue;
          const int n = nodes[u];
          f[13 + 3 * u] = (V[n][0] * tx + V[n][1] * ty) * hl;
          f[14 + 3 * u] = (-V[n][0] * ty + V[n][1] * tx) * hl;
          f[15 + 3 * u] = V[n][2] * hl;
        }
        if (k == 1) f[22] = th[j];
        f[23] = lam[j][k] * lsc;
      }
      uint32_t pk[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        __nv_bfloat162 b2 = __floats2bfloat162_rn(f[2 * c], f[2 * c + 1]);
        pk[c] = *reinterpret_cast<uint32_t*>(&b2);
      }
      uint4* dst = reinterpret_cast<uint4*>(A.feat + ((size_t)(S.fb + i) * 6 + k) * 32);
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
    }
  }
}

// One step of the chamber law of Sec. V-A (Eq. 11-12) towards the target t: inflating
// adds p_s k_i ((t - p) / p_s)^2, deflating removes min(p k_d, T_p), never past t.
__device__ __forceinline__ float chamber_law(float p, float t, const SolverArgs& A) {
  if (t > p) {
    const float dp = (t - p) / A.p_s;
    return fminf(t, p + A.p_s * dp * dp * A.k_i);
  }
  if (t < p) return fmaxf(t, p - fminf(p * A.k_d, A.t_p));
  return p;
}

// Newton + PCR solve of one contact-free substep (see pcr.cuh) for the snake of this lane
// group, from the current multipliers and displacements; returns the final normalised
// residual and the number of matrix-vector products.
template <int NPL, int G>
__device__ void newton_pcr(const SnakeK& S, const SolverArgs& A, int q, bool valid,
                           const float (&xs)[NPL][3], float (&dx)[NPL][3], float (&lam)[NPL][6],
                           const float (&th)[NPL], float* smem, float& r_end, int& mv) {
  const int lane = threadIdx.x & 31;
  const PcrSmem M = pcr_smem(smem, NPL);
  const int base = (lane / G) * G * NPL;
  const float L0 = S.L0;
  float x[NPL][3], z[NPL][3], p[NPL][3], qv[NPL][3], iD[NPL][3], y[NPL][3], u[NPL][3];
  bool gdone = !valid;
  mv = 0;
  r_end = 0.f;
  for (;;) {
    // ---- linearise at x = x_s + d: segments, rows, preconditioner, right-hand side
#pragma unroll
    for (int j = 0; j < NPL; ++j)
#pragma unroll
      for (int d = 0; d < 3; ++d) { M.U(d, base + q * NPL + j) = xs[j][d]; M.U(3 + d, base + q * NPL + j) = dx[j][d]; }
    __syncwarp();
    float r = 0.f;
    Seg sp = make_seg(1.f, 0.f, 0.f, L0);
    {
      const int i0 = q * NPL, s0 = base + i0;
      if (valid && i0 >= 1 && i0 <= S.N - 1)
        sp = make_seg((M.U(0, s0) - M.U(0, s0 - 1)) + (M.U(3, s0) - M.U(3, s0 - 1)),
                      (M.U(1, s0) - M.U(1, s0 - 1)) + (M.U(4, s0) - M.U(4, s0 - 1)),
                      (M.U(2, s0) - M.U(2, s0 - 1)) + (M.U(5, s0) - M.U(5, s0 - 1)), L0);
    }
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = q * NPL + j, s = base + i;
      const bool act = valid && i < S.N;
      const float wi = (i < S.nfix) ? 0.f : S.inv_m;
      const float wl = (i - 1 < S.nfix) ? 0.f : S.inv_m;
      const float wr = (i + 1 < S.nfix) ? 0.f : S.inv_m;
      const bool has_seg = act && i + 1 <= S.N - 1;
      Seg sc = make_seg(1.f, 0.f, 0.f, L0);
      if (has_seg)
        sc = make_seg((M.U(0, s + 1) - xs[j][0]) + (M.U(3, s + 1) - dx[j][0]),
                      (M.U(1, s + 1) - xs[j][1]) + (M.U(4, s + 1) - dx[j][1]),
                      (M.U(2, s + 1) - xs[j][2]) + (M.U(5, s + 1) - dx[j][2]), L0);
      // segment i's gradients for the products (zero where there is no segment)
      M.S(0, s) = has_seg ? sc.nx : 0.f; M.S(1, s) = has_seg ? sc.ny : 0.f; M.S(2, s) = has_seg ? sc.nz : 0.f;
      M.S(3, s) = has_seg ? sc.gyx : 0.f; M.S(4, s) = has_seg ? sc.gyy : 0.f;
      M.S(5, s) = has_seg ? sc.gpx : 0.f; M.S(6, s) = has_seg ? sc.gpy : 0.f; M.S(7, s) = has_seg ? sc.gpz : 0.f;
      float b[3] = {0.f, 0.f, 0.f};
      iD[j][0] = iD[j][1] = iD[j][2] = 0.f;
      if (has_seg && wi + wr > 0.f) {  // stretch
        const float c = sc.len - L0;
        r = fmaxf(r, fabsf(c + S.at_s * lam[j][0]) * S.inv_L0);
        iD[j][0] = 1.f / (wi + wr + S.at_s);
        b[0] = -(c + S.at_s * lam[j][0]);
      }
      if (act && i >= 1 && i <= S.N - 2) {
        {  // yaw
          const float cz = sp.ex * sc.ey - sp.ey * sc.ex, dh = sp.ex * sc.ex + sp.ey * sc.ey;
          const float c = L0 * (atan2_bend(cz, dh) - th[j]);
          const float g1x = -sp.gyx - sc.gyx, g1y = -sp.gyy - sc.gyy;
          const float wg = wl * (sp.gyx * sp.gyx + sp.gyy * sp.gyy) + wi * (g1x * g1x + g1y * g1y) +
                           wr * (sc.gyx * sc.gyx + sc.gyy * sc.gyy);
          if (wg > 0.f) {
            r = fmaxf(r, fabsf(c + S.at_b * lam[j][1]) * S.inv_L0);
            iD[j][1] = 1.f / (wg + S.at_b);
            b[1] = -(c + S.at_b * lam[j][1]);
          }
        }
        {  // pitch
          const float c = L0 * (sc.beta - sp.beta);
          const float g1x = -sp.gpx - sc.gpx, g1y = -sp.gpy - sc.gpy, g1z = -sp.gpz - sc.gpz;
          const float wg = wl * (sp.gpx * sp.gpx + sp.gpy * sp.gpy + sp.gpz * sp.gpz) +
                           wi * (g1x * g1x + g1y * g1y + g1z * g1z) +
                           wr * (sc.gpx * sc.gpx + sc.gpy * sc.gpy + sc.gpz * sc.gpz);
          if (wg > 0.f) {
            r = fmaxf(r, fabsf(c + S.at_b * lam[j][2]) * S.inv_L0);
            iD[j][2] = 1.f / (wg + S.at_b);
            b[2] = -(c + S.at_b * lam[j][2]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) { x[j][k] = 0.f; z[j][k] = b[k] * iD[j][k]; p[j][k] = z[j][k]; }
      sp = sc;
    }
    if (!(r <= 3.0e38f)) r = INFINITY;
    r = group_max<G>(r);
    __syncwarp();
    if (!gdone && (r <= A.tol || mv >= A.K)) { gdone = true; r_end = r; }
    if (__all_sync(kFull, gdone)) break;
    // ---- PCR on (J M^-1 J^T + alpha~) dlambda = b, diagonal preconditioner, from 0
    pcr_matvec<NPL>(S, M, q, base, valid, iD, z, y, u);
    if (!gdone) ++mv;
    float zaz = 0.f;
#pragma unroll
    for (int j = 0; j < NPL; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) { qv[j][k] = y[j][k]; zaz += z[j][k] * y[j][k]; }
    zaz = group_sum<G>(zaz);
    bool on = !gdone;
    for (int it = 0; it < A.pcr_iters; ++it) {
      bool go = on && mv < A.K;
      if (!__any_sync(kFull, go)) break;
      float qs = 0.f;
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) qs += qv[j][k] * qv[j][k] * iD[j][k];
      qs = group_sum<G>(qs);
      if (go && !(qs > 0.f)) { on = false; go = false; }
      const float alpha = go ? zaz / qs : 0.f;
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) { x[j][k] += alpha * p[j][k]; z[j][k] -= alpha * qv[j][k] * iD[j][k]; }
      pcr_matvec<NPL>(S, M, q, base, valid, iD, z, y, u);
      if (go) ++mv;
      float zaz2 = 0.f;
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) zaz2 += z[j][k] * y[j][k];
      zaz2 = group_sum<G>(zaz2);
      const float beta = (go && zaz != 0.f) ? zaz2 / zaz : 0.f;
      if (go) zaz = zaz2;
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (!go) continue;
          p[j][k] = z[j][k] + beta * p[j][k];
          qv[j][k] = y[j][k] + beta * qv[j][k];
        }
    }
    // ---- lambda += dlambda, d += M^-1 J^T dlambda (gradients at the linearisation point)
#pragma unroll
    for (int j = 0; j < NPL; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) M.V(k, base + q * NPL + j) = x[j][k];
    __syncwarp();
    pcr_jt<NPL>(S, M, q, base, valid, u);
    __syncwarp();
    if (!gdone) {
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        if (q * NPL + j >= S.N) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) { lam[j][k] += x[j][k]; dx[j][k] += u[j][k]; }
      }
    }
  }
}

// Advances the snake owned by this lane group.  Fused mode (A.split == 0): A.n_steps
// env-steps with all substeps in registers.  Split mode: finishes substep A.sub (if >= 0)
// of the current env-step and the substeps after it up to A.sub + A.span - 1, then, if
// the next one exists, begins it (gait, filter, prediction), writes its features and
// leaves the state in HBM at that point (positions = substep start, velocities =
// predicted), so that the warm-start network can run between two launches.
// VAR: which solve the kernel carries.  kVarJacobi: the Jacobi relaxation with isotropic
// friction; kVarAniso: the same with the anisotropic friction path (batches where some
// snake has mu_side > 0; the other kernels carry none of its code); kVarPcr: Newton +
// preconditioned conjugate residual over the bilateral rows (contact-free substeps;
// `smem` is its per-block shared-memory area).
enum { kVarJacobi = 0, kVarAniso = 1, kVarPcr = 2 };
template <int NPL, int G, bool SPLIT, int VAR>
__device__ void run_group(const SolverArgs& A, int snake, bool valid, float* smem) {
  constexpr bool ANISO = VAR == kVarAniso;
  const int lane = threadIdx.x & 31;
  const int q = lane & (G - 1);
  SnakeK S;
  SnakeParams P;
  if (valid) P = A.prm[snake];
  else { P = SnakeParams(); P.n_links = 0; P.seg_per_link = 1; P.mass = 1.f; P.L0 = 1.f;
         P.tau_inf = 1.f; P.tau_def = 1.f; }
  const float h = A.h;
  S.N = valid ? P.n_links * P.seg_per_link + 1 : 0;
  S.seg = P.seg_per_link; S.nfix = P.n_fixed; S.L = P.n_links;
  S.nb = valid ? A.node_off[snake] : 0;
  S.fb = valid ? A.feat_off[snake] : 0;
  S.lb = valid ? A.link_off[snake] : 0;
  S.L0 = P.L0; S.inv_L0 = 1.0f / P.L0; S.inv_m = 1.0f / P.mass; S.mass = P.mass;
  S.at_s = P.alpha_s / (h * h); S.at_b = P.alpha_b / (h * h);
  S.mu = P.mu; S.radius = P.radius; S.gain = P.gain;
  S.mu_side = P.mu_side > 0.f ? P.mu_side : 0.f;
  S.inv_mu = S.mu_side > 0.f ? 1.0f / P.mu : 0.f;
  S.inv_mu_side = S.mu_side > 0.f ? 1.0f / S.mu_side : 0.f;
  S.e_inf = expf(-h / P.tau_inf); S.e_def = expf(-h / P.tau_def);
  S.om_m = A.omega * S.mass;
  S.damp_over_h = expf(-P.damping * h) / h;

  // x = xs + dx; between substeps dx holds the last substep's displacement
  float xs[NPL][3], dx[NPL][3], v[NPL][3], lam[NPL][6], pR[NPL], pL[NPL], th[NPL];
  const bool mid = SPLIT && A.sub >= 0;  // HBM holds a begun substep
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = q * NPL + j;
    th[j] = 0.f;
    dx[j][0] = dx[j][1] = dx[j][2] = 0.f;
    if (valid && i < S.N) {
      const float4 p = A.pos[S.nb + i];
      const float4 u = A.vel[S.nb + i];
      xs[j][0] = p.x; xs[j][1] = p.y; xs[j][2] = p.z;
      v[j][0] = u.x; v[j][1] = u.y; v[j][2] = u.z;
#pragma unroll
      for (int k = 0; k < 6; ++k) lam[j][k] = A.lam[(size_t)(S.nb + i) * 6 + k];
      const int kl = min(i / S.seg, S.L - 1);
      const float2 pp = A.press[S.lb + kl];
      pR[j] = pp.x; pL[j] = pp.y;
      if (mid) {
        if (i >= S.nfix) { dx[j][0] = h * v[j][0]; dx[j][1] = h * v[j][1]; dx[j][2] = h * v[j][2]; }
        th[j] = (i % S.seg == 0) ? 0.f : S.gain * (pR[j] - pL[j]) * S.L0;
      }
    } else {
      xs[j][0] = xs[j][1] = xs[j][2] = 0.f;
      v[j][0] = v[j][1] = v[j][2] = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) lam[j][k] = 0.f;
      pR[j] = pL[j] = 0.f;
    }
  }

  // (a1) gait target at the end of substep s, (a2) chamber latency, (a3) rest angle,
  // (a4) predict: the substep starts at x = xs + dx; dx restarts at h v
  auto begin_substep = [&](long long step, int s) {
    // first-order model: target at the end of the substep, every substep; the law of
    // Sec. V-A: once per law step, target at the end of the law step, held in between
    const long long gsub = step * A.n_sub + s;
    const bool law = A.latency == SIM_LATENCY_LAW;
    const bool move = !law || gsub % A.law_every == 0;
    const double tp = (double)(law ? gsub + A.law_every : gsub + 1) * A.h_d;
    double cyc = (double)P.gait_freq * tp;
    cyc -= floor(cyc);
    const float phase = 6.283185307179586f * (float)cyc;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = q * NPL + j;
      if (!(valid && i < S.N)) continue;
      const int kl = min(i / S.seg, S.L - 1);
      if (move) {
        float u;
        if (A.ucmd) {
          u = A.ucmd[S.lb + kl];
        } else {
          // argument reduced to [-pi, pi] first, where the fast sine is accurate to ~1e-6
          float arg = phase + (float)kl * P.gait_lag;
          arg -= 6.283185307179586f * rintf(arg * 0.15915494309189535f);
          float a = P.gait_offset + P.gait_scale * __sinf(arg);
          a = fminf(1.f, fmaxf(-1.f, a)) * P.gait_amp;
          if (P.gait_alternate != 0.f && (kl & 1)) a = -a;
          u = a;
        }
        const float tR = fmaxf(u, 0.f), tL = fmaxf(-u, 0.f);
        if (law) {
          pR[j] = chamber_law(pR[j], tR, A);
          pL[j] = chamber_law(pL[j], tL, A);
        } else {
          pR[j] = tR + (pR[j] - tR) * (tR > pR[j] ? S.e_inf : S.e_def);
          pL[j] = tL + (pL[j] - tL) * (tL > pL[j] ? S.e_inf : S.e_def);
        }
      }
      th[j] = (i % S.seg == 0) ? 0.f : S.gain * (pR[j] - pL[j]) * S.L0;
    }
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = q * NPL + j;
      xs[j][0] += dx[j][0]; xs[j][1] += dx[j][1]; xs[j][2] += dx[j][2];
      dx[j][0] = dx[j][1] = dx[j][2] = 0.f;
      if (valid && i < S.N && i >= S.nfix) {
        v[j][0] += h * A.g[0]; v[j][1] += h * A.g[1]; v[j][2] += h * A.g[2];
        dx[j][0] = h * v[j][0]; dx[j][1] = h * v[j][1]; dx[j][2] = h * v[j][2];
      }
    }
  };

  // warm start, (a5, a6) Jacobi iterations, (a7) velocity with damping; `net`: the learned
  // warm start adds the network's prediction at this substep
  auto finish_substep = [&](float& rmax, int& itot, bool net) {
    float xsl[3], xsr[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xsl[d] = __shfl_up_sync(kFull, xs[NPL - 1][d], 1, G);
      xsr[d] = __shfl_down_sync(kFull, xs[0][d], 1, G);
    }
    bool stop;
    if (A.warm == 0) {
#pragma unroll
      for (int j = 0; j < NPL; ++j)
#pragma unroll
        for (int k = 0; k < 6; ++k) lam[j][k] = 0.f;
    } else {
      // warm start: beta lambda_prev, or beta_net lambda_prev + m g h^2 y on the rows the
      // network predicts at this substep
      const float sc = S.mass * 9.81f * h * h;
#pragma unroll
      for (int j = 0; j < NPL; ++j) {
        const int i = q * NPL + j;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const bool pk = A.warm == 2 && net && A.lam0 && valid && i < S.N &&
                          (A.net_rows == SIM_NET_ROWS_ALL || k < (A.net_rows == SIM_NET_ROWS_BILATERAL ? 3 : 1));
          float l = (pk ? A.beta_net : A.beta) * lam[j][k];
          if (pk) l += A.lam0[(size_t)(S.fb + i) * 6 + k] * sc;
          lam[j][k] = l;
        }
      }
      row_pass<NPL, G, true, ANISO>(S, A, q, valid, 0, xs, dx, xsl, xsr, lam, th, stop);
    }
    bool done = !valid;
    float rs = 0.f;
    int ks = 0;
    if (VAR == kVarPcr) {
      newton_pcr<NPL, G>(S, A, q, valid, xs, dx, lam, th, smem, rs, ks);
    } else {
      for (int k = 0;; ++k) {
        const float r = row_pass<NPL, G, false, ANISO>(S, A, q, !done, k, xs, dx, xsl, xsr, lam, th, stop);
        if (!done && stop) { done = true; rs = r; ks = k; }
        if (__all_sync(kFull, done)) break;
      }
    }
    // a non-finite displacement anywhere in the snake marks the step (fmaxf drops NaN)
    float bad = 0.f;
#pragma unroll
    for (int j = 0; j < NPL; ++j)
      if (!(fabsf(dx[j][0]) + fabsf(dx[j][1]) + fabsf(dx[j][2]) <= 3.0e38f)) bad = 1.f;
    bad = group_max<G>(bad);
    rmax = fmaxf(rmax, rs);
    if (!(rs <= 3.0e38f) || bad > 0.f) rmax = INFINITY;
    itot += ks;
#pragma unroll
    for (int j = 0; j < NPL; ++j) {
      const int i = q * NPL + j;
      if (valid && i < S.N && i >= S.nfix) {
        v[j][0] = dx[j][0] * S.damp_over_h;
        v[j][1] = dx[j][1] * S.damp_over_h;
        v[j][2] = dx[j][2] * S.damp_over_h;
      } else {
        v[j][0] = v[j][1] = v[j][2] = 0.f;
      }
    }
  };

  const long long step0 = *A.step_dev;
  float rmax = 0.f;
  int itot = 0;
  bool at_boundary = true;  // state ends at a substep boundary (x = xs + dx, v)
  if (!SPLIT) {
    for (int st = 0; st < A.n_steps; ++st) {
      rmax = 0.f;
      itot = 0;
      for (int s = 0; s < A.n_sub; ++s) {
        begin_substep(step0 + st, s);
        finish_substep(rmax, itot, false);
      }
    }
  } else {
    if (A.sub > 0 && valid && q == 0) { rmax = A.resid[snake]; itot = A.iters[snake]; }
    // the substep begun by the previous launch, then the rest of the span in full (one
    // call site, so that the kernel carries one copy of the pass)
    int next = A.sub + 1;
    for (int t = A.sub; t >= 0 && t < A.sub + A.span && t < A.n_sub; ++t) {
      if (t > A.sub) begin_substep(step0, t);
      finish_substep(rmax, itot, t % A.net_every == 0);
      next = t + 1;
    }
    if (next < A.n_sub) {
      begin_substep(step0, next);
      if (SPLIT) write_features<NPL, G>(S, A, q, valid, xs, dx, v, lam, th);
      at_boundary = false;
    }
  }
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const int i = q * NPL + j;
    if (i >= S.N) continue;
    const float wi = (i < S.nfix) ? 0.f : S.inv_m;
    if (at_boundary)
      A.pos[S.nb + i] = make_float4(xs[j][0] + dx[j][0], xs[j][1] + dx[j][1], xs[j][2] + dx[j][2], wi);
    else
      A.pos[S.nb + i] = make_float4(xs[j][0], xs[j][1], xs[j][2], wi);
    A.vel[S.nb + i] = make_float4(v[j][0], v[j][1], v[j][2], 0.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) A.lam[(size_t)(S.nb + i) * 6 + k] = lam[j][k];
    if (i % S.seg == 0 && i / S.seg < S.L) A.press[S.lb + i / S.seg] = make_float2(pR[j], pL[j]);
  }
  if (q == 0 && (!SPLIT || A.sub >= 0)) {
    A.resid[snake] = rmax;
    A.iters[snake] = itot;
    int st = 0;
    if (!(rmax <= 3.0e38f)) st = -4;               // SIM_ENAN
    else if (A.tol > 0.f && rmax > A.tol) st = 1;  // SIM_NOT_CONVERGED
    A.status[snake] = st;
  }
}

}  // namespace snakesim
