// Reverse-mode adjoint of the executed solver map, for calibration.
//
// The map differentiated is the one the calibration runs execute: every substep starts
// cold (lambda = 0) and applies exactly K Jacobi updates, so the map is a fixed
// composition of the gait / latency filter (Eq. 9, Sec. III), the rest angle (Eq. 3-4),
// the prediction, K relaxations of Eq. 8 and the damped velocity update; clamps and the
// Coulomb projection contribute the derivative of the branch they took.  Parameters per
// snake: theta = (alpha_b, damping d, tau_inflate, tau_deflate, gain G); loss gradient
// arrives as d L / d tip(t) for the last node after every env-step.
//
// One warp owns one snake (one CTA per snake); node and row arrays live in shared memory
// and the lanes stride over nodes, with __syncthreads() between phases.  The backward pass
// of a checkpoint segment recomputes the segment's substep-start states, then walks the
// substeps in reverse; inside a substep it recomputes the K iterates (stored in an
// L2-resident scratch) and runs the transposed iteration:
//   delta^_j = lambda^_j + sum_i w_i g_ji . x^_i,   g^_ji = w_i delta_j x^_i,
//   through the row update (bilateral, contact clamp, friction projection) to c^, lambda^,
//   alpha~^ and D^, then  x^ += sum_j g_j c^_j + H_j g^_j  with the Hessians of the
//   stretch, heading (atan2) and elevation (atan2(z, rho)) rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "snakesim.h"

namespace {

constexpr float kPiF = 3.14159265358979f;

struct AdjArgs {
  const SnakeParams* prm;
  const float* theta;     // [S][5] alpha_b, damping, tau_inf, tau_def, gain
  const int* node_off;    // [S + 1]
  const int* link_off;    // [S + 1]
  int n_snakes, n_max, l_max;
  // working state (segment start in, segment end out) [S][n_max*3] / [S][l_max*2]
  float* x;
  float* v;
  float* p;
  // substep-start records of a segment [S][n_rec][...]
  float* rec_x;
  float* rec_v;
  float* rec_p;
  int n_rec;              // capacity in substeps
  // iterates scratch [S][K + 1][n_max * 9]
  float* iters;
  // tips [n_total_steps][S][3] (forward) / their adjoint (backward)
  float* tips;
  const float* tips_bar;
  int tip_base;           // global env-step index of the segment's first step
  // adjoint carried between segments [S][n_max*3], [S][n_max*3], [S][l_max*2]; grad [S][5]
  float* xb;
  float* vb;
  float* pb;
  float* grad;
  float inv_T;            // unused scale hook (the loss scale is in tips_bar)
  long long step0;        // env-step counter at the segment start
  int n_steps;            // env-steps in the segment
  int store;              // forward: record substep starts
  int n_sub, K, contact;
  float h, omega, g[3];
  double h_d;
};

struct Snk {
  int N, L, seg, nfix;
  float L0, m, w, as, ab, G, ti, td, mu, d, r, amp, freq, lag, off, scale, alt;
};

struct Sh {  // shared-memory arrays of one snake
  float *xs, *X, *v, *p, *pin, *th, *lam, *c, *D, *dl, *lnew, *g, *aux;
  int* br;
  float *xb, *vb, *pb, *lb, *gb, *cb, *dbar, *lbn, *xn, *xsb, *thb;
};

// Threads per snake (one block per snake): the lanes stride over the snake's nodes and
// rows, and the phases of a substep are separated by block barriers.
constexpr int kAdjThreads = 64;
__device__ __forceinline__ int tid() { return threadIdx.x; }

__device__ Snk load_snake(const AdjArgs& A, int s) {
  const SnakeParams P = A.prm[s];
  const float* th = A.theta + 5 * s;
  Snk S;
  S.L = P.n_links; S.seg = P.seg_per_link; S.N = S.L * S.seg + 1; S.nfix = P.n_fixed;
  S.L0 = P.L0; S.m = P.mass; S.w = 1.f / P.mass; S.as = P.alpha_s;
  S.ab = th[0]; S.d = th[1]; S.ti = th[2]; S.td = th[3]; S.G = th[4];
  S.mu = P.mu; S.r = P.radius; S.amp = P.gait_amp; S.freq = P.gait_freq; S.lag = P.gait_lag;
  S.off = P.gait_offset; S.scale = P.gait_scale; S.alt = P.gait_alternate;
  return S;
}

__device__ __forceinline__ float wnode(const Snk& S, int i) { return i < S.nfix ? 0.f : S.w; }
__device__ __forceinline__ float* G3(const Sh& M, int i, int k, int l) { return M.g + ((i * 6 + k) * 3 + l) * 3; }
__device__ __forceinline__ float* GB3(const Sh& M, int i, int k, int l) { return M.gb + ((i * 6 + k) * 3 + l) * 3; }
__device__ __forceinline__ bool row_on(const Snk& S, const AdjArgs& A, int i, int k) {
  if (k == 0) return i <= S.N - 2;
  if (k <= 2) return i >= 1 && i <= S.N - 2;
  return A.contact != 0;
}
__device__ __forceinline__ int row_nodes(int k) { return k == 0 ? 2 : (k <= 2 ? 3 : 1); }
__device__ __forceinline__ int row_node(int i, int k, int l) { return k == 0 ? i + l : (k <= 2 ? i - 1 + l : i); }

__device__ __forceinline__ float gait(const Snk& S, int k, double t) {
  double cyc = (double)S.freq * t;
  cyc -= floor(cyc);
  float a = S.off + S.scale * sinf(2.f * kPiF * (float)cyc + (float)k * S.lag);
  a = fminf(1.f, fmaxf(-1.f, a)) * S.amp;
  if (S.alt != 0.f && (k & 1)) a = -a;
  return a;
}

__device__ __forceinline__ void psi_grad(const float* e, float* g) {
  const float h2 = e[0] * e[0] + e[1] * e[1];
  g[0] = -e[1] / h2; g[1] = e[0] / h2; g[2] = 0.f;
}
__device__ __forceinline__ void psi_hess_vec(const float* e, const float* u, float* o) {
  const float h2 = e[0] * e[0] + e[1] * e[1], h4 = h2 * h2;
  const float a = 2.f * e[0] * e[1] / h4, b = (e[1] * e[1] - e[0] * e[0]) / h4;
  o[0] = a * u[0] + b * u[1]; o[1] = b * u[0] - a * u[1]; o[2] = 0.f;
}
__device__ __forceinline__ void beta_grad(const float* e, float* g) {
  const float rho2 = e[0] * e[0] + e[1] * e[1], rho = sqrtf(rho2), r2 = rho2 + e[2] * e[2];
  g[0] = -e[2] * e[0] / (rho * r2); g[1] = -e[2] * e[1] / (rho * r2); g[2] = rho / r2;
}
__device__ __forceinline__ void beta_hess_vec(const float* e, const float* u, float* o) {
  const float x = e[0], y = e[1], z = e[2];
  const float rho2 = x * x + y * y, rho = sqrtf(rho2), r2 = rho2 + z * z, r4 = r2 * r2;
  const float q = rho * r2, dq = r2 / rho + 2.f * rho, q2 = q * q;
  const float fxx = -z / q + z * x * x * dq / q2, fxy = z * x * y * dq / q2;
  const float fxz = -x / q + 2.f * z * z * x / (rho * r4);
  const float fyy = -z / q + z * y * y * dq / q2, fyz = -y / q + 2.f * z * z * y / (rho * r4);
  const float fzx = x / (rho * r2) - 2.f * rho * x / r4, fzy = y / (rho * r2) - 2.f * rho * y / r4;
  const float fzz = -2.f * rho * z / r4;
  o[0] = fxx * u[0] + fxy * u[1] + fxz * u[2];
  o[1] = fxy * u[0] + fyy * u[1] + fyz * u[2];
  o[2] = fzx * u[0] + fzy * u[1] + fzz * u[2];
}

// (a1-a3) gait, latency filter, rest angles of substep s of env-step `step`.  M.pin keeps
// the pressures before the filter.
__device__ void begin_pressure(const Snk& S, const AdjArgs& A, long long step, int s, const Sh& M) {
  const double t = ((double)step * A.n_sub + (double)(s + 1)) * A.h_d;
  for (int k = tid(); k < S.L; k += kAdjThreads) {
    const float a = gait(S, k, t);
    const float tg[2] = {fmaxf(a, 0.f), fmaxf(-a, 0.f)};
    for (int c = 0; c < 2; ++c) {
      const float pp = M.p[2 * k + c];
      M.pin[2 * k + c] = pp;
      const float tau = tg[c] > pp ? S.ti : S.td;
      M.p[2 * k + c] = tg[c] + (pp - tg[c]) * expf(-A.h / tau);
    }
  }
  __syncthreads();
  for (int i = tid(); i < S.N; i += kAdjThreads) {
    float th = 0.f;
    if (i >= 1 && i <= S.N - 2 && i % S.seg != 0) {
      const int k = i / S.seg;
      th = S.G * (M.p[2 * k] - M.p[2 * k + 1]) * S.L0;
    }
    M.th[i] = th;
  }
  __syncthreads();
}

// rows of every node at (X, lam): values, gradients, diagonal, relaxed update, branches
__device__ void eval_rows(const Snk& S, const AdjArgs& A, const Sh& M) {
  const float h2 = A.h * A.h;
  for (int i = tid(); i < S.N; i += kAdjThreads) {
    for (int k = 0; k < 6; ++k) {
      const int j = i * 6 + k;
      M.c[j] = 0.f; M.D[j] = 0.f; M.dl[j] = 0.f; M.lnew[j] = M.lam[j]; M.br[j] = 0;
      for (int q = 0; q < 9; ++q) M.g[j * 9 + q] = 0.f;
    }
    const float* X = M.X;
    if (i <= S.N - 2) {
      float e[3];
      for (int d = 0; d < 3; ++d) e[d] = X[3 * (i + 1) + d] - X[3 * i + d];
      const float len = sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      M.c[i * 6] = len - S.L0;
      for (int d = 0; d < 3; ++d) { G3(M, i, 0, 0)[d] = -e[d] / len; G3(M, i, 0, 1)[d] = e[d] / len; }
    }
    if (i >= 1 && i <= S.N - 2) {
      float e1[3], e2[3], a[3], b[3];
      for (int d = 0; d < 3; ++d) { e1[d] = X[3 * i + d] - X[3 * (i - 1) + d]; e2[d] = X[3 * (i + 1) + d] - X[3 * i + d]; }
      const float cz = e1[0] * e2[1] - e1[1] * e2[0], dh = e1[0] * e2[0] + e1[1] * e2[1];
      M.c[i * 6 + 1] = S.L0 * (atan2f(cz, dh) - M.th[i]);
      psi_grad(e1, a); psi_grad(e2, b);
      for (int d = 0; d < 3; ++d) {
        G3(M, i, 1, 0)[d] = S.L0 * a[d]; G3(M, i, 1, 1)[d] = -S.L0 * (a[d] + b[d]); G3(M, i, 1, 2)[d] = S.L0 * b[d];
      }
      const float b1 = atan2f(e1[2], sqrtf(e1[0] * e1[0] + e1[1] * e1[1]));
      const float b2 = atan2f(e2[2], sqrtf(e2[0] * e2[0] + e2[1] * e2[1]));
      M.c[i * 6 + 2] = S.L0 * (b2 - b1);
      beta_grad(e1, a); beta_grad(e2, b);
      for (int d = 0; d < 3; ++d) {
        G3(M, i, 2, 0)[d] = S.L0 * a[d]; G3(M, i, 2, 1)[d] = -S.L0 * (a[d] + b[d]); G3(M, i, 2, 2)[d] = S.L0 * b[d];
      }
    }
    if (A.contact) {
      M.c[i * 6 + 3] = X[3 * i + 2] - S.r; G3(M, i, 3, 0)[2] = 1.f;
      M.c[i * 6 + 4] = X[3 * i] - M.xs[3 * i]; G3(M, i, 4, 0)[0] = 1.f;
      M.c[i * 6 + 5] = X[3 * i + 1] - M.xs[3 * i + 1]; G3(M, i, 5, 0)[1] = 1.f;
    }
    for (int k = 0; k < 6; ++k) {
      if (!row_on(S, A, i, k)) continue;
      float sum = 0.f;
      for (int l = 0; l < row_nodes(k); ++l) {
        const float* g = G3(M, i, k, l);
        sum += wnode(S, row_node(i, k, l)) * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
      }
      M.D[i * 6 + k] = sum;
    }
    for (int k = 0; k < 3; ++k) {
      const int j = i * 6 + k;
      if (!row_on(S, A, i, k) || M.D[j] == 0.f) continue;
      const float at = (k == 0 ? S.as : S.ab) / h2;
      const float dl = A.omega * (-M.c[j] - at * M.lam[j]) / (M.D[j] + at);
      M.dl[j] = dl; M.lnew[j] = M.lam[j] + dl;
    }
    const float wi = wnode(S, i);
    if (A.contact && wi > 0.f) {
      const int j = i * 6 + 3, jx = j + 1, jy = j + 2;
      const float tmp = M.lam[j] + A.omega * (-M.c[j] * S.m);
      M.br[j] = tmp > 0.f;
      M.lnew[j] = fmaxf(0.f, tmp); M.dl[j] = M.lnew[j] - M.lam[j];
      const float tx = M.lam[jx] - A.omega * M.c[jx] * S.m, ty = M.lam[jy] - A.omega * M.c[jy] * S.m;
      const float rad = S.mu * M.lam[j];
      float nx = tx, ny = ty;
      int br = 0;
      if (tx * tx + ty * ty > rad * rad) {
        if (rad <= 0.f) { nx = ny = 0.f; br = 2; }
        else { const float n = sqrtf(tx * tx + ty * ty); nx = tx * rad / n; ny = ty * rad / n; br = 1; }
      }
      M.br[jx] = br; M.aux[3 * i] = tx; M.aux[3 * i + 1] = ty; M.aux[3 * i + 2] = rad;
      M.lnew[jx] = nx; M.lnew[jy] = ny; M.dl[jx] = nx - M.lam[jx]; M.dl[jy] = ny - M.lam[jy];
    }
  }
  __syncthreads();
}

// x_i += w_i sum_j g_ji dl_j (fixed order), lambda <- lambda_new
__device__ void apply_rows(const Snk& S, const AdjArgs& A, const Sh& M) {
  for (int i = tid(); i < S.N; i += kAdjThreads) {
    const int list[11][3] = {{i - 1, 0, 1}, {i, 0, 0}, {i - 1, 1, 2}, {i - 1, 2, 2}, {i, 1, 1}, {i, 2, 1},
                             {i + 1, 1, 0}, {i + 1, 2, 0}, {i, 3, 0}, {i, 4, 0}, {i, 5, 0}};
    float acc[3] = {0.f, 0.f, 0.f};
    for (int q = 0; q < 11; ++q) {
      const int o = list[q][0], k = list[q][1], l = list[q][2];
      if (o < 0 || o >= S.N || !row_on(S, A, o, k)) continue;
      const float* g = G3(M, o, k, l);
      const float dd = M.dl[o * 6 + k];
      for (int d = 0; d < 3; ++d) acc[d] += g[d] * dd;
    }
    const float wi = wnode(S, i);
    for (int d = 0; d < 3; ++d) M.X[3 * i + d] += wi * acc[d];
    for (int k = 0; k < 6; ++k) M.lam[i * 6 + k] = M.lnew[i * 6 + k];
  }
  __syncthreads();
}

// One substep forward from (M.X = x, M.v, M.p).  With `it`, stores the K + 1 iterates.
__device__ void substep_fwd(const Snk& S, const AdjArgs& A, long long step, int s, const Sh& M, float* it) {
  begin_pressure(S, A, step, s, M);
  const float h = A.h;
  for (int i = tid(); i < S.N; i += kAdjThreads)
    for (int d = 0; d < 3; ++d) {
      M.xs[3 * i + d] = M.X[3 * i + d];
      if (i >= S.nfix) { M.v[3 * i + d] += h * A.g[d]; M.X[3 * i + d] += h * M.v[3 * i + d]; }
    }
  for (int i = tid(); i < S.N * 6; i += kAdjThreads) M.lam[i] = 0.f;
  __syncthreads();
  for (int k = 0; k < A.K; ++k) {
    if (it) {
      float* dst = it + (size_t)k * A.n_max * 9;
      for (int i = tid(); i < S.N * 3; i += kAdjThreads) dst[i] = M.X[i];
      for (int i = tid(); i < S.N * 6; i += kAdjThreads) dst[A.n_max * 3 + i] = M.lam[i];
    }
    eval_rows(S, A, M);
    apply_rows(S, A, M);
  }
  if (it) {
    float* dst = it + (size_t)A.K * A.n_max * 9;
    for (int i = tid(); i < S.N * 3; i += kAdjThreads) dst[i] = M.X[i];
  }
  const float cd = expf(-S.d * h) / h;
  for (int i = tid(); i < S.N; i += kAdjThreads)
    for (int d = 0; d < 3; ++d)
      M.v[3 * i + d] = i >= S.nfix ? (M.X[3 * i + d] - M.xs[3 * i + d]) * cd : 0.f;
  __syncthreads();
}

// Adjoint of one substep.  On entry M.xb, M.vb, M.pb hold the adjoints of the substep's
// output (x, v, p) and M.X, M.v, M.p its start state; on exit they hold the adjoints of
// its input.  tb[5] (per lane) accumulates the parameter adjoints.
__device__ void substep_adj(const Snk& S, const AdjArgs& A, long long step, int s, const Sh& M,
                            float* it, float* tb) {
  const float h = A.h, h2 = h * h;
  const float om = A.omega;
  // start state -> keep copies of the inputs the adjoint needs (pressures before filter)
  substep_fwd(S, A, step, s, M, it);  // M.pin: filter inputs; M.p: filtered; M.xs: start x
  const float* XK = it + (size_t)A.K * A.n_max * 9;
  const float cd = expf(-S.d * h) / h;
  for (int i = tid(); i < S.N; i += kAdjThreads)
    for (int d = 0; d < 3; ++d) {
      M.xsb[3 * i + d] = 0.f;
      if (i >= S.nfix) {
        const float gv = M.vb[3 * i + d];
        M.xb[3 * i + d] += gv * cd;
        M.xsb[3 * i + d] -= gv * cd;
        tb[1] += gv * (XK[3 * i + d] - M.xs[3 * i + d]) * (-h) * cd;
      }
    }
  for (int i = tid(); i < S.N * 6; i += kAdjThreads) M.lb[i] = 0.f;
  for (int i = tid(); i < S.N; i += kAdjThreads) M.thb[i] = 0.f;
  __syncthreads();
  for (int k = A.K - 1; k >= 0; --k) {
    const float* src = it + (size_t)k * A.n_max * 9;
    for (int i = tid(); i < S.N * 3; i += kAdjThreads) M.X[i] = src[i];
    for (int i = tid(); i < S.N * 6; i += kAdjThreads) M.lam[i] = src[A.n_max * 3 + i];
    __syncthreads();
    eval_rows(S, A, M);
    // delta^ and g^ from x^(k+1), lambda^(k+1)
    for (int o = tid(); o < S.N; o += kAdjThreads)
      for (int kk = 0; kk < 6; ++kk) {
        const int j = o * 6 + kk;
        for (int q = 0; q < 9; ++q) M.gb[j * 9 + q] = 0.f;
        M.cb[j] = 0.f;
        if (!row_on(S, A, o, kk)) { M.dbar[j] = 0.f; continue; }
        float db = M.lb[j];
        for (int l = 0; l < row_nodes(kk); ++l) {
          const int n = row_node(o, kk, l);
          const float wn = wnode(S, n);
          const float* g = G3(M, o, kk, l);
          float* gbp = GB3(M, o, kk, l);
          for (int d = 0; d < 3; ++d) {
            db += wn * g[d] * M.xb[3 * n + d];
            gbp[d] += wn * M.dl[j] * M.xb[3 * n + d];
          }
        }
        M.dbar[j] = db;
      }
    __syncthreads();
    // through the row updates
    for (int o = tid(); o < S.N; o += kAdjThreads) {
      for (int kk = 0; kk < 6; ++kk) M.lbn[o * 6 + kk] = M.lb[o * 6 + kk];
      for (int kk = 0; kk < 3; ++kk) {
        const int j = o * 6 + kk;
        if (!row_on(S, A, o, kk) || M.D[j] == 0.f) continue;
        const float at = (kk == 0 ? S.as : S.ab) / h2, Dt = M.D[j] + at;
        const float dlb = om * M.dbar[j], dlv = M.dl[j] / om;
        M.cb[j] += -dlb / Dt;
        M.lbn[j] += -at * dlb / Dt;
        const float Db = -dlv * dlb / Dt;
        const float atb = -M.lam[j] * dlb / Dt + Db;
        if (kk >= 1) tb[0] += atb / h2;
        for (int l = 0; l < row_nodes(kk); ++l) {
          const float wn = wnode(S, row_node(o, kk, l));
          const float* g = G3(M, o, kk, l);
          float* gbp = GB3(M, o, kk, l);
          for (int d = 0; d < 3; ++d) gbp[d] += 2.f * wn * g[d] * Db;
        }
        if (kk == 1) M.thb[o] += -S.L0 * M.cb[j];
      }
      const float wo = wnode(S, o);
      if (A.contact && wo > 0.f) {
        const int j = o * 6 + 3, jx = j + 1, jy = j + 2;
        const float newb = M.dbar[j];
        M.lbn[j] -= newb;
        const float tmpb = M.br[j] ? newb : 0.f;
        M.lbn[j] += tmpb;
        M.cb[j] += -om * tmpb * S.m;
        const float nbx = M.dbar[jx], nby = M.dbar[jy];
        M.lbn[jx] -= nbx; M.lbn[jy] -= nby;
        float tbx = 0.f, tby = 0.f;
        const int br = M.br[jx];
        if (br == 0) { tbx = nbx; tby = nby; }
        else if (br == 1) {
          const float tx = M.aux[3 * o], ty = M.aux[3 * o + 1], rad = M.aux[3 * o + 2];
          const float n = sqrtf(tx * tx + ty * ty), ux = tx / n, uy = ty / n;
          const float dot = ux * nbx + uy * nby;
          tbx = rad / n * (nbx - ux * dot); tby = rad / n * (nby - uy * dot);
          M.lbn[j] += S.mu * dot;
        }
        M.lbn[jx] += tbx; M.lbn[jy] += tby;
        M.cb[jx] += -om * tbx * S.m; M.cb[jy] += -om * tby * S.m;
      }
    }
    __syncthreads();
    // x^k adjoint: x^(k+1) adjoint + sum_j g_j c^_j + H_j g^_j, gathered per node
    for (int i = tid(); i < S.N; i += kAdjThreads) {
      float acc[3] = {M.xb[3 * i], M.xb[3 * i + 1], M.xb[3 * i + 2]};
      const int list[11][3] = {{i - 1, 0, 1}, {i, 0, 0}, {i - 1, 1, 2}, {i - 1, 2, 2}, {i, 1, 1}, {i, 2, 1},
                               {i + 1, 1, 0}, {i + 1, 2, 0}, {i, 3, 0}, {i, 4, 0}, {i, 5, 0}};
      for (int q = 0; q < 11; ++q) {
        const int o = list[q][0], kk = list[q][1], l = list[q][2];
        if (o < 0 || o >= S.N || !row_on(S, A, o, kk)) continue;
        const float* g = G3(M, o, kk, l);
        const float cbv = M.cb[o * 6 + kk];
        for (int d = 0; d < 3; ++d) acc[d] += g[d] * cbv;
      }
      // Hessian terms: stretch rows (i-1, i) and (i, i+1); bend rows centred on i-1, i, i+1
      for (int o = i - 1; o <= i; ++o) {  // stretch owned by o connects o, o+1
        if (o < 0 || o > S.N - 2) continue;
        float e[3], u[3];
        for (int d = 0; d < 3; ++d) {
          e[d] = M.X[3 * (o + 1) + d] - M.X[3 * o + d];
          u[d] = GB3(M, o, 0, 1)[d] - GB3(M, o, 0, 0)[d];
        }
        const float len = sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        const float dot = (e[0] * u[0] + e[1] * u[1] + e[2] * u[2]) / len;
        const float sg = (o == i) ? -1.f : 1.f;  // node o gets -q, node o+1 gets +q
        for (int d = 0; d < 3; ++d) acc[d] += sg * (u[d] - e[d] / len * dot) / len;
      }
      for (int o = i - 1; o <= i + 1; ++o) {
        if (o < 1 || o > S.N - 2) continue;
        float e1[3], e2[3];
        for (int d = 0; d < 3; ++d) { e1[d] = M.X[3 * o + d] - M.X[3 * (o - 1) + d]; e2[d] = M.X[3 * (o + 1) + d] - M.X[3 * o + d]; }
        for (int kk = 1; kk <= 2; ++kk) {
          float u1[3], u2[3], A1[3], A2[3];
          for (int d = 0; d < 3; ++d) {
            u1[d] = S.L0 * (GB3(M, o, kk, 0)[d] - GB3(M, o, kk, 1)[d]);
            u2[d] = S.L0 * (GB3(M, o, kk, 2)[d] - GB3(M, o, kk, 1)[d]);
          }
          if (kk == 1) { psi_hess_vec(e1, u1, A1); psi_hess_vec(e2, u2, A2); }
          else { beta_hess_vec(e1, u1, A1); beta_hess_vec(e2, u2, A2); }
          // node o-1: -A1; node o: A1 - A2; node o+1: +A2
          for (int d = 0; d < 3; ++d) {
            if (i == o - 1) acc[d] -= A1[d];
            else if (i == o) acc[d] += A1[d] - A2[d];
            else acc[d] += A2[d];
          }
        }
      }
      M.xn[3 * i] = acc[0]; M.xn[3 * i + 1] = acc[1]; M.xn[3 * i + 2] = acc[2];
      if (A.contact) {  // friction rows measure x - x_start
        M.xsb[3 * i] -= M.cb[i * 6 + 4];
        M.xsb[3 * i + 1] -= M.cb[i * 6 + 5];
      }
    }
    __syncthreads();
    for (int i = tid(); i < S.N * 3; i += kAdjThreads) M.xb[i] = M.xn[i];
    for (int i = tid(); i < S.N * 6; i += kAdjThreads) M.lb[i] = M.lbn[i];
    __syncthreads();
  }
  // prediction: x0 = x_in + h v1 (free), v1 = v_in + h g
  for (int i = tid(); i < S.N; i += kAdjThreads)
    for (int d = 0; d < 3; ++d) {
      const float x0b = M.xb[3 * i + d];
      M.xb[3 * i + d] = x0b + M.xsb[3 * i + d];
      M.vb[3 * i + d] = i >= S.nfix ? h * x0b : 0.f;
    }
  __syncthreads();
  // rest angles theta = G (p_R' - p_L') L0 and the latency filter
  if (tid() == 0) {
    for (int i = 1; i <= S.N - 2; ++i) {
      if (i % S.seg == 0) continue;
      const int k = i / S.seg;
      const float t = M.thb[i];
      tb[4] += t * (M.p[2 * k] - M.p[2 * k + 1]) * S.L0;
      M.pb[2 * k] += t * S.G * S.L0;
      M.pb[2 * k + 1] -= t * S.G * S.L0;
    }
  }
  __syncthreads();
  const double tt = ((double)step * A.n_sub + (double)(s + 1)) * A.h_d;
  for (int k = tid(); k < S.L; k += kAdjThreads) {
    const float a = gait(S, k, tt);
    const float tg[2] = {fmaxf(a, 0.f), fmaxf(-a, 0.f)};
    for (int c = 0; c < 2; ++c) {
      const float pp = M.pin[2 * k + c];
      const bool inf = tg[c] > pp;
      const float tau = inf ? S.ti : S.td, e = expf(-h / tau);
      const float g = M.pb[2 * k + c];
      M.pb[2 * k + c] = g * e;
      tb[inf ? 2 : 3] += g * (pp - tg[c]) * e * h / (tau * tau);
    }
  }
  __syncthreads();
}

__device__ Sh carve(uint8_t* base, int n, int l) {
  float* f = reinterpret_cast<float*>(base);
  Sh M;
  auto take = [&](int cnt) { float* p = f; f += cnt; return p; };
  M.xs = take(3 * n); M.X = take(3 * n); M.v = take(3 * n); M.p = take(2 * l); M.pin = take(2 * l);
  M.th = take(n); M.lam = take(6 * n); M.c = take(6 * n); M.D = take(6 * n); M.dl = take(6 * n);
  M.lnew = take(6 * n); M.g = take(54 * n); M.aux = take(3 * n);
  M.br = reinterpret_cast<int*>(take(6 * n));
  M.xb = take(3 * n); M.vb = take(3 * n); M.pb = take(2 * l); M.lb = take(6 * n); M.gb = take(54 * n);
  M.cb = take(6 * n); M.dbar = take(6 * n); M.lbn = take(6 * n); M.xn = take(3 * n); M.xsb = take(3 * n);
  M.thb = take(n);
  return M;
}

}  // namespace

size_t adjoint_smem_bytes(int n_max, int l_max) {
  return sizeof(float) * (size_t)(3 * n_max * 3 + 2 * l_max * 3 + n_max * 2 + 6 * n_max * 10 +
                                  54 * n_max * 2 + 3 * n_max * 5);
}

// Forward over a segment: state in A.x/A.v/A.p (per snake), tips written, substep starts
// recorded when A.store.
__global__ void __launch_bounds__(kAdjThreads) adj_forward_kernel(AdjArgs A) {
  const int s = blockIdx.x;
  if (s >= A.n_snakes) return;
  extern __shared__ __align__(16) uint8_t smem[];
  const Snk S = load_snake(A, s);
  Sh M = carve(smem, A.n_max, A.l_max);
  float* gx = A.x + (size_t)s * A.n_max * 3;
  float* gv = A.v + (size_t)s * A.n_max * 3;
  float* gp = A.p + (size_t)s * A.l_max * 2;
  for (int i = tid(); i < S.N * 3; i += kAdjThreads) { M.X[i] = gx[i]; M.v[i] = gv[i]; }
  for (int i = tid(); i < S.L * 2; i += kAdjThreads) M.p[i] = gp[i];
  __syncthreads();
  for (int st = 0; st < A.n_steps; ++st) {
    for (int sb = 0; sb < A.n_sub; ++sb) {
      if (A.store) {
        const size_t q = (size_t)s * A.n_rec + (size_t)st * A.n_sub + sb;
        for (int i = tid(); i < S.N * 3; i += kAdjThreads) {
          A.rec_x[q * A.n_max * 3 + i] = M.X[i];
          A.rec_v[q * A.n_max * 3 + i] = M.v[i];
        }
        for (int i = tid(); i < S.L * 2; i += kAdjThreads) A.rec_p[q * A.l_max * 2 + i] = M.p[i];
      }
      substep_fwd(S, A, A.step0 + st, sb, M, nullptr);
    }
    if (A.tips && tid() == 0) {
      float* t = A.tips + ((size_t)(A.tip_base + st) * A.n_snakes + s) * 3;
      t[0] = M.X[3 * (S.N - 1)]; t[1] = M.X[3 * (S.N - 1) + 1]; t[2] = M.X[3 * (S.N - 1) + 2];
    }
    __syncthreads();
  }
  for (int i = tid(); i < S.N * 3; i += kAdjThreads) { gx[i] = M.X[i]; gv[i] = M.v[i]; }
  for (int i = tid(); i < S.L * 2; i += kAdjThreads) gp[i] = M.p[i];
}

// Backward over a segment whose substep starts were recorded; adjoints carried in
// A.xb/A.vb/A.pb, parameter adjoints added to A.grad.
__global__ void __launch_bounds__(kAdjThreads) adj_backward_kernel(AdjArgs A) {
  const int s = blockIdx.x;
  if (s >= A.n_snakes) return;
  extern __shared__ __align__(16) uint8_t smem[];
  const Snk S = load_snake(A, s);
  Sh M = carve(smem, A.n_max, A.l_max);
  float* gxb = A.xb + (size_t)s * A.n_max * 3;
  float* gvb = A.vb + (size_t)s * A.n_max * 3;
  float* gpb = A.pb + (size_t)s * A.l_max * 2;
  float* it = A.iters + (size_t)s * (A.K + 1) * A.n_max * 9;
  for (int i = tid(); i < S.N * 3; i += kAdjThreads) { M.xb[i] = gxb[i]; M.vb[i] = gvb[i]; }
  for (int i = tid(); i < S.L * 2; i += kAdjThreads) M.pb[i] = gpb[i];
  __syncthreads();
  float tb[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int st = A.n_steps - 1; st >= 0; --st) {
    if (tid() == 0) {
      const float* t = A.tips_bar + ((size_t)(A.tip_base + st) * A.n_snakes + s) * 3;
      for (int d = 0; d < 3; ++d) M.xb[3 * (S.N - 1) + d] += t[d];
    }
    __syncthreads();
    for (int sb = A.n_sub - 1; sb >= 0; --sb) {
      const size_t q = (size_t)s * A.n_rec + (size_t)st * A.n_sub + sb;
      for (int i = tid(); i < S.N * 3; i += kAdjThreads) {
        M.X[i] = A.rec_x[q * A.n_max * 3 + i];
        M.v[i] = A.rec_v[q * A.n_max * 3 + i];
      }
      for (int i = tid(); i < S.L * 2; i += kAdjThreads) M.p[i] = A.rec_p[q * A.l_max * 2 + i];
      __syncthreads();
      substep_adj(S, A, A.step0 + st, sb, M, it, tb);
    }
  }
  for (int i = tid(); i < S.N * 3; i += kAdjThreads) { gxb[i] = M.xb[i]; gvb[i] = M.vb[i]; }
  for (int i = tid(); i < S.L * 2; i += kAdjThreads) gpb[i] = M.pb[i];
  // parameter adjoints: a butterfly in every warp, then the warps' sums in a fixed order
  __shared__ float part[kAdjThreads / 32][5];
  for (int k = 0; k < 5; ++k) {
    float v = tb[k];
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((tid() & 31) == 0) part[tid() / 32][k] = v;
  }
  __syncthreads();
  if (tid() == 0)
    for (int k = 0; k < 5; ++k) {
      float v = 0.f;
      for (int w = 0; w < kAdjThreads / 32; ++w) v += part[w][k];
      A.grad[5 * s + k] += v;
    }
}

// ------------------------------------------------------------------ host side
namespace snakesim {

struct CalibState {
  int n_snakes = 0, n_max = 0, l_max = 0, n_sub = 0, K = 0, contact = 0, ckpt = 0, n_steps = 0;
  long long step0 = 0;
  float h = 0.f, omega = 0.f, g[3] = {0.f, 0.f, 0.f};
  double h_d = 0.0;
  size_t smem = 0;
  // device
  float *theta = nullptr, *x = nullptr, *v = nullptr, *p = nullptr;
  float *ck_x = nullptr, *ck_v = nullptr, *ck_p = nullptr;  // [n_ckpt][S][...]
  float *rec_x = nullptr, *rec_v = nullptr, *rec_p = nullptr, *iters = nullptr;
  float *xb = nullptr, *vb = nullptr, *pb = nullptr;
  int n_ckpt = 0, n_rec = 0;
  // allocated sizes (floats) of the buffers above, in the same order: buffers grow when a
  // run needs more and are otherwise kept from call to call (no allocation, and no
  // free, on the path of a repeated run)
  size_t cap[14] = {};
  float** slot(int i) {
    float** ptrs[] = {&theta, &x, &v, &p, &ck_x, &ck_v, &ck_p, &rec_x, &rec_v, &rec_p, &iters, &xb, &vb, &pb};
    return ptrs[i];
  }
  cudaError_t grow(int i, size_t n) {
    if (n <= cap[i]) return cudaSuccess;
    float** q = slot(i);
    if (*q) cudaFree(*q);
    *q = nullptr;
    cap[i] = 0;
    cudaError_t e = cudaMalloc(q, n * sizeof(float));
    if (e == cudaSuccess) cap[i] = n;
    return e;
  }
  void release() {
    for (int i = 0; i < 14; ++i) if (*slot(i)) cudaFree(*slot(i));
    *this = CalibState();
  }
};
enum { kTheta, kX, kV, kP, kCkX, kCkV, kCkP, kRecX, kRecV, kRecP, kIters, kXb, kVb, kPb };

}  // namespace snakesim

using snakesim::CalibState;

namespace {
__global__ void gather_state_kernel(const float4* pos, const float4* vel, const float2* press,
                                    const int* node_off, const int* link_off, int n_snakes, int n_max,
                                    int l_max, float* x, float* v, float* p) {
  const int s = blockIdx.x;
  if (s >= n_snakes) return;
  const int nb = node_off[s], N = node_off[s + 1] - nb, lb = link_off[s], L = link_off[s + 1] - lb;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float4 a = pos[nb + i], b = vel[nb + i];
    float* xd = x + ((size_t)s * n_max + i) * 3;
    float* vd = v + ((size_t)s * n_max + i) * 3;
    xd[0] = a.x; xd[1] = a.y; xd[2] = a.z;
    vd[0] = b.x; vd[1] = b.y; vd[2] = b.z;
  }
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const float2 q = press[lb + k];
    p[((size_t)s * l_max + k) * 2] = q.x;
    p[((size_t)s * l_max + k) * 2 + 1] = q.y;
  }
}

__global__ void scatter_state_kernel(float4* pos, float4* vel, float2* press, const int* node_off,
                                     const int* link_off, int n_snakes, int n_max, int l_max,
                                     const float* x, const float* v, const float* p, const SnakeParams* prm) {
  const int s = blockIdx.x;
  if (s >= n_snakes) return;
  const int nb = node_off[s], N = node_off[s + 1] - nb, lb = link_off[s], L = link_off[s + 1] - lb;
  const float w = 1.f / prm[s].mass;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float* xd = x + ((size_t)s * n_max + i) * 3;
    const float* vd = v + ((size_t)s * n_max + i) * 3;
    pos[nb + i] = make_float4(xd[0], xd[1], xd[2], i < prm[s].n_fixed ? 0.f : w);
    vel[nb + i] = make_float4(vd[0], vd[1], vd[2], 0.f);
  }
  for (int k = threadIdx.x; k < L; k += blockDim.x)
    press[lb + k] = make_float2(p[((size_t)s * l_max + k) * 2], p[((size_t)s * l_max + k) * 2 + 1]);
}
}  // namespace

namespace snakesim {

#define ACU(call)                                                    \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) { err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return e_ == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA; } \
  } while (0)

AdjArgs make_adj(const CalibState& C, const SnakeParams* prm, const int* no, const int* lo) {
  AdjArgs A = {};
  A.prm = prm; A.theta = C.theta; A.node_off = no; A.link_off = lo;
  A.n_snakes = C.n_snakes; A.n_max = C.n_max; A.l_max = C.l_max;
  A.x = C.x; A.v = C.v; A.p = C.p;
  A.rec_x = C.rec_x; A.rec_v = C.rec_v; A.rec_p = C.rec_p; A.n_rec = C.n_rec;
  A.iters = C.iters; A.xb = C.xb; A.vb = C.vb; A.pb = C.pb;
  A.n_sub = C.n_sub; A.K = C.K; A.contact = C.contact; A.h = C.h; A.h_d = C.h_d; A.omega = C.omega;
  A.g[0] = C.g[0]; A.g[1] = C.g[1]; A.g[2] = C.g[2];
  return A;
}

SimStatus calib_forward(CalibState& C, const SnakeParams* prm, const int* no, const int* lo, int n_snakes,
                        int n_max, int l_max, const float* theta, int n_steps, int ckpt, long long step0,
                        int n_sub, int K, int contact, double dt, float omega, const float* gvec,
                        float4* pos4, float4* vel4, float2* press2, float* tips, cudaStream_t st,
                        std::string& err) {
  C.n_snakes = n_snakes; C.n_max = n_max; C.l_max = l_max; C.n_sub = n_sub; C.K = K; C.contact = contact;
  C.ckpt = ckpt; C.n_steps = n_steps; C.step0 = step0; C.h_d = dt / n_sub; C.h = (float)C.h_d;
  C.omega = omega; C.g[0] = gvec[0]; C.g[1] = gvec[1]; C.g[2] = gvec[2];
  C.n_ckpt = (n_steps + ckpt - 1) / ckpt;
  C.n_rec = ckpt * n_sub;
  const size_t S = n_snakes, xs = S * n_max * 3, ps = S * l_max * 2;
  ACU(C.grow(kTheta, S * 5));
  ACU(C.grow(kX, xs));
  ACU(C.grow(kV, xs));
  ACU(C.grow(kP, ps));
  ACU(C.grow(kCkX, C.n_ckpt * xs));
  ACU(C.grow(kCkV, C.n_ckpt * xs));
  ACU(C.grow(kCkP, C.n_ckpt * ps));
  ACU(cudaMemcpyAsync(C.theta, theta, S * 5 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  C.smem = adjoint_smem_bytes(n_max, l_max);
  ACU(cudaFuncSetAttribute(adj_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem));
  ACU(cudaFuncSetAttribute(adj_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C.smem));
  gather_state_kernel<<<n_snakes, 128, 0, st>>>(pos4, vel4, press2, no, lo, n_snakes, n_max, l_max, C.x, C.v, C.p);
  ACU(cudaGetLastError());
  for (int c = 0; c < C.n_ckpt; ++c) {
    ACU(cudaMemcpyAsync(C.ck_x + c * xs, C.x, xs * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ACU(cudaMemcpyAsync(C.ck_v + c * xs, C.v, xs * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ACU(cudaMemcpyAsync(C.ck_p + c * ps, C.p, ps * sizeof(float), cudaMemcpyDeviceToDevice, st));
    AdjArgs A = make_adj(C, prm, no, lo);
    A.tips = tips;
    A.tip_base = c * ckpt;
    A.step0 = step0 + (long long)c * ckpt;
    A.n_steps = std::min(ckpt, n_steps - c * ckpt);
    A.store = 0;
    adj_forward_kernel<<<n_snakes, kAdjThreads, C.smem, st>>>(A);
    ACU(cudaGetLastError());
  }
  scatter_state_kernel<<<n_snakes, 128, 0, st>>>(pos4, vel4, press2, no, lo, n_snakes, n_max, l_max, C.x, C.v, C.p, prm);
  ACU(cudaGetLastError());
  return SIM_OK;
}

SimStatus calib_backward(CalibState& C, const SnakeParams* prm, const int* no, const int* lo,
                         const float* tips_bar, float* grad, cudaStream_t st, std::string& err) {
  if (C.n_steps <= 0) { err = "no calibration forward pass to differentiate"; return SIM_EINVAL; }
  const size_t S = C.n_snakes, xs = S * C.n_max * 3, ps = S * C.l_max * 2;
  ACU(C.grow(kRecX, S * C.n_rec * C.n_max * 3));
  ACU(C.grow(kRecV, S * C.n_rec * C.n_max * 3));
  ACU(C.grow(kRecP, S * C.n_rec * C.l_max * 2));
  ACU(C.grow(kIters, S * (C.K + 1) * C.n_max * 9));
  ACU(C.grow(kXb, xs));
  ACU(C.grow(kVb, xs));
  ACU(C.grow(kPb, ps));
  ACU(cudaMemsetAsync(C.xb, 0, xs * sizeof(float), st));
  ACU(cudaMemsetAsync(C.vb, 0, xs * sizeof(float), st));
  ACU(cudaMemsetAsync(C.pb, 0, ps * sizeof(float), st));
  ACU(cudaMemsetAsync(grad, 0, S * 5 * sizeof(float), st));
  for (int c = C.n_ckpt - 1; c >= 0; --c) {
    ACU(cudaMemcpyAsync(C.x, C.ck_x + c * xs, xs * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ACU(cudaMemcpyAsync(C.v, C.ck_v + c * xs, xs * sizeof(float), cudaMemcpyDeviceToDevice, st));
    ACU(cudaMemcpyAsync(C.p, C.ck_p + c * ps, ps * sizeof(float), cudaMemcpyDeviceToDevice, st));
    AdjArgs A = make_adj(C, prm, no, lo);
    A.tip_base = c * C.ckpt;
    A.step0 = C.step0 + (long long)c * C.ckpt;
    A.n_steps = std::min(C.ckpt, C.n_steps - c * C.ckpt);
    A.store = 1;
    A.tips = nullptr;
    adj_forward_kernel<<<C.n_snakes, kAdjThreads, C.smem, st>>>(A);
    ACU(cudaGetLastError());
    A.store = 0;
    A.tips_bar = tips_bar;
    A.grad = grad;
    adj_backward_kernel<<<C.n_snakes, kAdjThreads, C.smem, st>>>(A);
    ACU(cudaGetLastError());
  }
  return SIM_OK;
}

CalibState* calib_new() { return new CalibState(); }
void calib_delete(CalibState* C) {
  if (C) { C->release(); delete C; }
}

}  // namespace snakesim
