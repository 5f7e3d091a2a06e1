// FP64 CPU oracle for the soft-snake compliant-constraint solve.
//
// TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the benchmark's
// CPU-baseline leg are the only callers; the product library never links or loads
// this file, and this file includes nothing from the product.
//
// What it computes (Gasoto et al., "A Validated Physical Model For Real-Time
// Simulation of Soft Robotic Snakes", arXiv 1904.02833):
//   * particles with lumped mass M_i = m 1_3                       (Sec. IV-A, Eq. 1)
//   * compliant bilateral constraints c_b(q, p) + E lambda_b = 0   (Sec. IV, equations of motion)
//   * pressure-driven actuation: the expanding chamber's rest length scales with
//     eps(p) = 1 + p/Y (Eq. 3-4); for a 1D chain with an inextensible centre layer
//     (Sec. V) this is a rest curvature linear in pressure, kappa = G (p_R - p_L)
//   * ground contact c_n = n^T (a - b) >= 0 (Eq. 7) with Coulomb friction limited to the
//     cone mu lambda_n (Sec. IV, equations of motion, last three lines)
//   * first-order implicit time stepping (Sec. IV-D); the Schur system of Eq. 8 is
//     relaxed with its own diagonal (the Jacobi preconditioner of Sec. IV-D): each row
//     gets  dlambda = (-c - alpha~ lambda) / (sum_i w_i |grad_i c|^2 + alpha~),
//     alpha~ = alpha / h^2, scaled by omega, applied to lambda and to x
//   * open-loop gait a_k = clamp(sin(w t + alpha k) + phi, -1, 1) A (Eq. 9, Sec. V-A),
//     antagonistic chambers (Sec. III), first-order inflate/deflate latency.
//
// The code is plain loops in the order the method states.  It is templated on the
// scalar type so that a forward-mode dual number carries derivatives with respect to
// five snake parameters through exactly the same code (used to check the adjoint).
//
// Parity pins (see tests/test_oracle_*.py): discrete circular arc under uniform
// pressure, small-deflection cantilever sag, pendulum period, momentum conservation,
// brute-force Newton on a 3-node chain, finite-difference constraint gradients,
// closed-form latency-filter step response, hand-computed gait and chamber-law values,
// Coulomb sliding distances (isotropic and anisotropic), a dense Schur solve for the
// Newton + PCR step, equivariance of whole env-steps under rotations about z, and the
// normalised residual on hand-built states whose value the definitions fix (every
// term: bilateral rows, the Fischer-Burmeister contact value, sticking and sliding
// friction pairs, rows on fixed nodes).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- scalars
inline double val(double a) { return a; }

// Forward-mode dual number with K directional derivatives.
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0.0) { for (int k = 0; k < K; ++k) d[k] = 0.0; }
  Dual(double a) : v(a) { for (int k = 0; k < K; ++k) d[k] = 0.0; }
};
template <int K> inline double val(const Dual<K>& a) { return a.v; }
template <int K> inline Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v + b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int K> inline Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v - b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int K> inline Dual<K> operator-(const Dual<K>& a) {
  Dual<K> r; r.v = -a.v; for (int k = 0; k < K; ++k) r.d[k] = -a.d[k]; return r; }
template <int K> inline Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v * b.v; for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int K> inline Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) {
  Dual<K> r; r.v = a.v / b.v;
  for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v);
  return r; }
template <int K> inline Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> inline Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> inline Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> inline Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> inline Dual<K> operator*(const Dual<K>& a, double b) { return a * Dual<K>(b); }
template <int K> inline Dual<K> operator*(double a, const Dual<K>& b) { return Dual<K>(a) * b; }
template <int K> inline Dual<K> operator/(const Dual<K>& a, double b) { return a / Dual<K>(b); }
template <int K> inline Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> inline Dual<K>& operator+=(Dual<K>& a, const Dual<K>& b) { a = a + b; return a; }
template <int K> inline Dual<K>& operator-=(Dual<K>& a, const Dual<K>& b) { a = a - b; return a; }
template <int K> inline Dual<K>& operator*=(Dual<K>& a, const Dual<K>& b) { a = a * b; return a; }
template <int K> inline Dual<K>& operator+=(Dual<K>& a, double b) { a.v += b; return a; }
template <int K> inline Dual<K> chain(const Dual<K>& a, double f, double df) {
  Dual<K> r; r.v = f; for (int k = 0; k < K; ++k) r.d[k] = df * a.d[k]; return r; }
template <int K> inline Dual<K> sqrt(const Dual<K>& a) { double s = std::sqrt(a.v); return chain(a, s, 0.5 / s); }
template <int K> inline Dual<K> exp(const Dual<K>& a) { double e = std::exp(a.v); return chain(a, e, e); }
template <int K> inline Dual<K> asin(const Dual<K>& a) {
  return chain(a, std::asin(a.v), 1.0 / std::sqrt(1.0 - a.v * a.v)); }
template <int K> inline Dual<K> fabs(const Dual<K>& a) { return a.v < 0 ? -a : a; }
template <int K> inline Dual<K> atan2(const Dual<K>& y, const Dual<K>& x) {
  Dual<K> r; double q = x.v * x.v + y.v * y.v; r.v = std::atan2(y.v, x.v);
  for (int k = 0; k < K; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) / q;
  return r; }

using std::sqrt; using std::exp; using std::asin; using std::atan2; using std::fabs;

template <class T> inline T tmax(const T& a, const T& b) { return val(a) >= val(b) ? a : b; }

template <class T> struct V3 { T x, y, z; };
template <class T> inline V3<T> sub(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline V3<T> scl(const V3<T>& a, const T& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// ---------------------------------------------------------------- layout
enum { P_L0, P_MASS, P_ALPHA_S, P_ALPHA_B, P_GAIN, P_TAU_INF, P_TAU_DEF, P_MU, P_DAMP,
       P_RADIUS, P_AMP, P_FREQ, P_LAG, P_OFFSET, P_SCALE, P_ALT, P_X0, P_Y0, P_Z0, P_YAW0,
       P_MU_SIDE, NPRM };
enum { C_DT, C_NSUB, C_ITERS, C_TOL, C_OMEGA, C_GX, C_GY, C_GZ, C_CONTACT, C_WARM, C_BETA,
       C_LATENCY, C_KI, C_KD, C_TP, C_PS, C_LAW_DT, C_SOLVER, C_PCR_ITERS, C_NET_ROWS, C_NET_EVERY,
       C_BETA_NET, NCFG };
// Row kinds; a node i owns one multiplier slot per kind: stretch (i, i+1), yaw and
// pitch bend centred on i, contact of i, friction of i along world x and y.
enum { R_STRETCH, R_YAW, R_PITCH, R_CONTACT, R_FX, R_FY, NK };
const double kPi = 3.14159265358979323846;

template <class T>
struct Snake {
  int N, L, seg, nfix;
  T L0, mass, alpha_s, alpha_b, gain, tau_inf, tau_def, mu, damp, radius;
  double amp, freq, lag, offset, scale, alt;
  double mu_side;  // > 0: anisotropic friction, mu along the body and mu_side across it
};

template <class T>
Snake<T> load_snake(const int* nl, const int* seg, const int* nfix, const double* prm, int s) {
  Snake<T> S;
  const double* p = prm + (size_t)s * NPRM;
  S.L = nl[s]; S.seg = seg[s]; S.N = S.L * S.seg + 1; S.nfix = nfix ? nfix[s] : 0;
  S.L0 = p[P_L0]; S.mass = p[P_MASS]; S.alpha_s = p[P_ALPHA_S]; S.alpha_b = p[P_ALPHA_B];
  S.gain = p[P_GAIN]; S.tau_inf = p[P_TAU_INF]; S.tau_def = p[P_TAU_DEF]; S.mu = p[P_MU];
  S.damp = p[P_DAMP]; S.radius = p[P_RADIUS];
  S.amp = p[P_AMP]; S.freq = p[P_FREQ]; S.lag = p[P_LAG]; S.offset = p[P_OFFSET];
  S.scale = p[P_SCALE]; S.alt = p[P_ALT]; S.mu_side = p[P_MU_SIDE];
  return S;
}

// Anisotropic friction (the wheels and scales of Sec. V): at node i the friction pair is
// limited to the ellipse (l_t / mu)^2 + (l_s / mu_side)^2 <= lambda_n^2 in the body frame
// (t along the chain at the substep start, s = z x t), instead of the disc of radius
// mu lambda_n.  Unit horizontal body tangent at node i from the substep-start positions.
template <class T>
void body_tangent(const std::vector<V3<T>>& XS, int N, int i, double& tx, double& ty) {
  const int a = std::max(i - 1, 0), b = std::min(i + 1, N - 1);
  const double ex = val(XS[b].x) - val(XS[a].x), ey = val(XS[b].y) - val(XS[a].y);
  const double n = std::sqrt(ex * ex + ey * ey);
  if (n > 0.0) { tx = ex / n; ty = ey / n; } else { tx = 1.0; ty = 0.0; }
}

// Projection of the pair (px, py) onto that ellipse with lambda_n = ln, radially in the
// coordinates scaled by the two coefficients (with mu_side = mu the disc projection).
template <class T>
void project_ellipse(T& px, T& py, double tx, double ty, double mu_t, double mu_s, const T& ln) {
  T a = px * tx + py * ty, b = py * tx - px * ty;  // along, across
  T u = a / mu_t, v = b / mu_s;
  const double r2 = val(u) * val(u) + val(v) * val(v);
  if (r2 > val(ln) * val(ln)) {
    if (val(ln) <= 0.0) { a = T(0.0); b = T(0.0); }
    else { T sc = ln / sqrt(u * u + v * v); a = a * sc; b = b * sc; }
  }
  px = a * tx - b * ty;
  py = a * ty + b * tx;
}

struct Cfg {
  double dt, h, tol, omega, g[3], beta;
  double beta_net;               // learned warm start: weight of lambda_prev under the prediction
  int n_sub, iters, contact, warm;
  int latency, law_every;        // chamber model (0 exponential, 1 Sec. V-A law), its period
  double k_i, k_d, t_p, p_s;     // Sec. V-A law: gains, deflation threshold, source pressure
  int solver, pcr_iters;         // 0 Jacobi; 1 Newton + preconditioned conjugate residual
  int net_rows, net_every;       // learned warm start: kinds predicted (0 all, 1 bilateral, 2 stretch), period
};
Cfg load_cfg(const double* c) {
  Cfg C;
  C.dt = c[C_DT]; C.n_sub = (int)c[C_NSUB]; C.h = C.dt / C.n_sub; C.iters = (int)c[C_ITERS];
  C.tol = c[C_TOL]; C.omega = c[C_OMEGA]; C.g[0] = c[C_GX]; C.g[1] = c[C_GY]; C.g[2] = c[C_GZ];
  C.contact = (int)c[C_CONTACT]; C.warm = (int)c[C_WARM]; C.beta = c[C_BETA];
  C.latency = (int)c[C_LATENCY]; C.k_i = c[C_KI]; C.k_d = c[C_KD]; C.t_p = c[C_TP]; C.p_s = c[C_PS];
  // the law's time step in whole substeps (at least one)
  C.law_every = std::max(1, (int)std::llround(c[C_LAW_DT] / C.h));
  C.solver = (int)c[C_SOLVER]; C.pcr_iters = (int)c[C_PCR_ITERS];
  C.net_rows = (int)c[C_NET_ROWS]; C.net_every = std::max(1, (int)c[C_NET_EVERY]);
  C.beta_net = c[C_BETA_NET] < 0.0 ? C.beta : c[C_BETA_NET];
  return C;
}

// One step of the chamber law of Sec. V-A (Eq. 11-12) towards the target p^: inflating
// (p^ > p) adds p_s dp^2 k_i with dp = (p^ - p) / p_s, deflating (p^ < p) removes
// min(p k_d, T_p); the valve stops at the target (clamp).
template <class T>
T chamber_law(const T& p, double tgt, const Cfg& C) {
  const double pv = val(p);
  if (tgt > pv) {
    T dp = (T(tgt) - p) / C.p_s;
    T q = p + C.p_s * dp * dp * C.k_i;
    return val(q) > tgt ? T(tgt) : q;
  }
  if (tgt < pv) {
    T dec = (pv * C.k_d < C.t_p) ? p * C.k_d : T(C.t_p);
    T q = p - dec;
    return val(q) < tgt ? T(tgt) : q;
  }
  return p;
}

// ---------------------------------------------------------------- gait (Eq. 9)
// a_k(t) = sigma_k * clamp(phi + s * sin(2 pi f t + k * lag), -1, 1) * A.
// The paper's form has s = 1 and sigma_k = 1 ("omega ... measured in Hz" is read as
// sin(2 pi f t)); s and the alternating sign sigma_k = (-1)^k generalise it so that a
// constant command (s = 0) and the alternating-sides gait use the same routine.
template <class T>
double gait_target(const Snake<T>& S, int k, double t) {
  double a = S.offset + S.scale * std::sin(2.0 * kPi * S.freq * t + k * S.lag);
  a = std::min(1.0, std::max(-1.0, a)) * S.amp;
  if (S.alt != 0.0 && (k & 1)) a = -a;
  return a;
}

// ---------------------------------------------------------------- constraint rows
// Row values and node gradients at the current positions.  Local node 0..2 of a bend
// row are (i-1, i, i+1); of a stretch row (i, i+1); per-node rows use local node 0.
template <class T>
struct Rows {
  int N;
  std::vector<T> c;            // [N][NK]
  std::vector<V3<T>> g;        // [N][NK][3]
  std::vector<char> on;        // row exists
  T& C(int i, int k) { return c[i * NK + k]; }
  V3<T>& G(int i, int k, int l) { return g[(i * NK + k) * 3 + l]; }
  char& ON(int i, int k) { return on[i * NK + k]; }
  void init(int n) {
    N = n; c.assign((size_t)n * NK, T(0.0)); g.assign((size_t)n * NK * 3, V3<T>{T(0.0), T(0.0), T(0.0)});
    on.assign((size_t)n * NK, 0);
  }
};

// Stretch: c = |x_{i+1} - x_i| - L0 (a distance constraint with constant rest length,
// Eq. 3 with eps = 1; Sec. V "structural" distance constraints).
template <class T>
void stretch_row(const V3<T>& xa, const V3<T>& xb, const T& L0, T& c, V3<T>* g) {
  V3<T> e = sub(xb, xa);
  T len = sqrt(dot(e, e));
  c = len - L0;
  V3<T> n = scl(e, T(1.0) / len);
  g[0] = scl(n, T(-1.0));
  g[1] = n;
}

// Bend rows are lengths, like every actuation row of Eq. 3: the bend angle times the
// segment rest length L0 (the displacement of the next node that the angle error
// amounts to).  With energy c^2 / (2 alpha_b) this is a rotational spring of stiffness
// L0^2 / alpha_b, i.e. a bending stiffness EI = L0^3 / alpha_b.
//
// Yaw bend: c = L0 (atan2(z . (e1 x e2), e1_h . e2_h) - theta_rest), e1 = x_i - x_{i-1},
// e2 = x_{i+1} - x_i, z the ground normal.  The gradient is the chain rule of atan2.
template <class T>
void yaw_row(const V3<T>& xa, const V3<T>& xb, const V3<T>& xc, const T& theta_rest,
             const T& L0, T& c, V3<T>* g) {
  V3<T> e1 = sub(xb, xa), e2 = sub(xc, xb);
  T cz = e1.x * e2.y - e1.y * e2.x;   // z . (e1 x e2)
  T dh = e1.x * e2.x + e1.y * e2.y;   // e1_h . e2_h
  c = L0 * (atan2(cz, dh) - theta_rest);
  T q = cz * cz + dh * dh;
  T a_cz = L0 * dh / q, a_dh = -L0 * cz / q;    // L0 d atan2 / d cz, L0 d atan2 / d dh
  // d cz / d e1 = (e2.y, -e2.x, 0),  d dh / d e1 = (e2.x, e2.y, 0)
  // d cz / d e2 = (-e1.y, e1.x, 0),  d dh / d e2 = (e1.x, e1.y, 0)
  V3<T> d1{a_cz * e2.y + a_dh * e2.x, -a_cz * e2.x + a_dh * e2.y, T(0.0)};
  V3<T> d2{-a_cz * e1.y + a_dh * e1.x, a_cz * e1.x + a_dh * e1.y, T(0.0)};
  g[0] = scl(d1, T(-1.0));
  g[1] = sub(d1, d2);
  g[2] = d2;
}

// Pitch bend: c = L0 (asin(e2_z / |e2|) - asin(e1_z / |e1|)) (rest value 0).
template <class T>
V3<T> elevation_grad(const V3<T>& e, T& beta) {
  T len2 = dot(e, e), len = sqrt(len2);
  T s = e.z / len;
  beta = asin(s);
  T f = T(1.0) / sqrt(T(1.0) - s * s);       // d asin / d s
  // d s / d e = z / |e| - e_z e / |e|^3
  V3<T> ds{-(e.z * e.x) / (len2 * len), -(e.z * e.y) / (len2 * len), T(1.0) / len - (e.z * e.z) / (len2 * len)};
  return scl(ds, f);
}
template <class T>
void pitch_row(const V3<T>& xa, const V3<T>& xb, const V3<T>& xc, const T& L0, T& c, V3<T>* g) {
  V3<T> e1 = sub(xb, xa), e2 = sub(xc, xb);
  T b1, b2;
  V3<T> d1 = scl(elevation_grad(e1, b1), L0), d2 = scl(elevation_grad(e2, b2), L0);
  c = L0 * (b2 - b1);
  // c depends on e1 with sign -1 and on e2 with sign +1
  g[0] = d1;                    // -(-d1): d e1 / d x_{i-1} = -1
  g[1] = sub(scl(d1, T(-1.0)), d2);
  g[2] = d2;
}

template <class T>
void eval_rows(const Snake<T>& S, const Cfg& C, const std::vector<V3<T>>& x,
               const std::vector<V3<T>>& xs, const std::vector<T>& theta_rest, Rows<T>& R) {
  const int N = S.N;
  for (int i = 0; i < N; ++i) {
    if (i < N - 1) {
      stretch_row(x[i], x[i + 1], S.L0, R.C(i, R_STRETCH), &R.G(i, R_STRETCH, 0));
      R.ON(i, R_STRETCH) = 1;
    }
    if (i >= 1 && i <= N - 2) {
      yaw_row(x[i - 1], x[i], x[i + 1], theta_rest[i], S.L0, R.C(i, R_YAW), &R.G(i, R_YAW, 0));
      pitch_row(x[i - 1], x[i], x[i + 1], S.L0, R.C(i, R_PITCH), &R.G(i, R_PITCH, 0));
      R.ON(i, R_YAW) = 1; R.ON(i, R_PITCH) = 1;
    }
    if (C.contact) {
      // Eq. 7 against the plane z = 0 with the node's contact radius r.
      R.C(i, R_CONTACT) = x[i].z - S.radius;
      R.G(i, R_CONTACT, 0) = V3<T>{T(0.0), T(0.0), T(1.0)};
      // Friction rows along the tangent basis D_i = [x, y] (Sec. IV): the tangential
      // displacement over the substep.
      R.C(i, R_FX) = x[i].x - xs[i].x;
      R.G(i, R_FX, 0) = V3<T>{T(1.0), T(0.0), T(0.0)};
      R.C(i, R_FY) = x[i].y - xs[i].y;
      R.G(i, R_FY, 0) = V3<T>{T(0.0), T(1.0), T(0.0)};
      R.ON(i, R_CONTACT) = R.ON(i, R_FX) = R.ON(i, R_FY) = 1;
    }
  }
}

// Node of local slot l of row kind k owned by node i.
inline int row_node(int i, int k, int l) {
  if (k == R_STRETCH) return i + l;
  if (k == R_YAW || k == R_PITCH) return i - 1 + l;
  return i;
}
inline int row_nodes(int k) { return k == R_STRETCH ? 2 : (k == R_YAW || k == R_PITCH) ? 3 : 1; }

template <class T>
T alpha_tilde(const Snake<T>& S, const Cfg& C, int k) {
  double h2 = C.h * C.h;
  if (k == R_STRETCH) return S.alpha_s / h2;
  if (k == R_YAW || k == R_PITCH) return S.alpha_b / h2;
  return T(0.0);
}

// sum_i w_i |grad_i c|^2 of a row (the diagonal of J M^-1 J^T, Sec. IV-D).
template <class T>
T row_wgrad2(Rows<T>& R, const std::vector<double>& w, int i, int k) {
  T s(0.0);
  for (int l = 0; l < row_nodes(k); ++l) {
    int n = row_node(i, k, l);
    V3<T>& g = R.G(i, k, l);
    s += w[n] * dot(g, g);
  }
  return s;
}

// Normalised residual of the solve, max over rows, every term a length divided by L0:
//  * bilateral rows: |c + alpha~ lambda|  (the compliant constraint c + E lambda = 0, Sec. IV)
//  * contact: |phi_FB(c_n, w lambda_n)| with the Fischer-Burmeister function
//    phi(a, b) = a + b - sqrt(a^2 + b^2), whose zeros are 0 <= a perp b >= 0 (Sec. IV-D)
//  * friction pair: |a - P_rho(a - u)|, a = w lambda_t, u = c_t the tangential
//    displacement, P_rho the projection onto the disc of radius rho = w mu lambda_n; it is
//    zero exactly when lambda_t sticks inside the cone (u = 0) or slides on its rim
//    opposite to u, and forces lambda_t = 0 when lambda_n = 0 (Sec. IV, Coulomb cone).
template <class T>
double residual(const Snake<T>& S, const Cfg& C, Rows<T>& R, const std::vector<double>& w,
                const std::vector<T>& lam, const std::vector<V3<T>>& XS) {
  double r = 0.0, L0 = val(S.L0);
  for (int i = 0; i < S.N; ++i) {
    for (int k = 0; k < NK; ++k) {
      if (!R.ON(i, k) || k == R_FY) continue;
      if (val(row_wgrad2(R, w, i, k)) == 0.0) continue;   // row on fixed nodes only
      double c = val(R.C(i, k)), l = val(lam[i * NK + k]), e = 0.0;
      if (k == R_STRETCH || k == R_YAW || k == R_PITCH) {
        e = std::fabs(c + val(alpha_tilde(S, C, k)) * l) / L0;
      } else if (k == R_CONTACT) {
        double b = w[i] * l;
        e = std::fabs(c + b - std::sqrt(c * c + b * b)) / L0;
      } else {  // friction pair of node i
        double ax = w[i] * val(lam[i * NK + R_FX]), ay = w[i] * val(lam[i * NK + R_FY]);
        double px = ax - val(R.C(i, R_FX)), py = ay - val(R.C(i, R_FY));
        if (S.mu_side > 0.0) {
          double tx, ty;
          body_tangent(XS, S.N, i, tx, ty);
          project_ellipse(px, py, tx, ty, val(S.mu), S.mu_side, w[i] * val(lam[i * NK + R_CONTACT]));
        } else {
          double rho = w[i] * val(S.mu) * val(lam[i * NK + R_CONTACT]);
          double n = std::sqrt(px * px + py * py);
          if (n > rho) {
            if (rho > 0.0) { px *= rho / n; py *= rho / n; } else { px = 0.0; py = 0.0; }
          }
        }
        e = std::sqrt((ax - px) * (ax - px) + (ay - py) * (ay - py)) / L0;
      }
      r = std::max(r, e);
    }
  }
  return r;
}

// x_i += w_i sum_j grad_i c_j d_j over the rows touching node i, summed in a fixed order:
// stretch(i-1), stretch(i), yaw/pitch(i-1), yaw/pitch(i), yaw/pitch(i+1), contact(i),
// friction x(i), friction y(i).
template <class T>
void apply_rows(int N, Rows<T>& R, const std::vector<double>& w, const std::vector<T>& d,
                std::vector<V3<T>>& X) {
  for (int i = 0; i < N; ++i) {
    if (w[i] == 0.0) continue;
    V3<T> acc{T(0.0), T(0.0), T(0.0)};
    auto add = [&](int owner, int kk, int l) {
      if (owner < 0 || owner >= N || !R.ON(owner, kk)) return;
      const V3<T>& g = R.G(owner, kk, l);
      const T& dd = d[owner * NK + kk];
      acc.x += g.x * dd; acc.y += g.y * dd; acc.z += g.z * dd;
    };
    add(i - 1, R_STRETCH, 1); add(i, R_STRETCH, 0);
    add(i - 1, R_YAW, 2); add(i - 1, R_PITCH, 2);
    add(i, R_YAW, 1); add(i, R_PITCH, 1);
    add(i + 1, R_YAW, 0); add(i + 1, R_PITCH, 0);
    add(i, R_CONTACT, 0); add(i, R_FX, 0); add(i, R_FY, 0);
    X[i].x += w[i] * acc.x; X[i].y += w[i] * acc.y; X[i].z += w[i] * acc.z;
  }
}

// ---------------------------------------------------------------- Newton + PCR
// The paper's own solve of a step (Sec. IV-D): Newton iterations on the compliant rows,
// each solving the Schur system of Eq. 8, (J M^-1 J^T + alpha~) dlambda = -(c + alpha~
// lambda), approximately with a fixed number of preconditioned conjugate residual (PCR)
// iterations with the diagonal (Jacobi) preconditioner, then lambda += dlambda and
// x += M^-1 J^T dlambda.  Bilateral rows only (stretch, yaw, pitch): the contact and
// friction rows of the paper's Fischer-Burmeister Newton are not part of this solver.
// Counts matrix-vector products with J M^-1 J^T (one per PCR iteration plus one per
// Newton step), stops when the normalised residual is <= tol or the count reaches `iters`.
template <class T>
int newton_pcr(const Snake<T>& S, const Cfg& C, std::vector<V3<T>>& X, const std::vector<V3<T>>& XS,
               const std::vector<T>& theta, Rows<T>& R, const std::vector<double>& w, std::vector<T>& lam,
               double& r_end) {
  const int N = S.N, n = N * NK;
  std::vector<T> D(n, T(1.0)), b(n, T(0.0)), x(n), z(n), p(n), q(n), Az(n);
  std::vector<char> act(n, 0);
  std::vector<V3<T>> U(N);
  auto dot_act = [&](const std::vector<T>& a, const std::vector<T>& c) {
    T s(0.0);
    for (int j = 0; j < n; ++j) if (act[j]) s += a[j] * c[j];
    return s;
  };
  // y = (J M^-1 J^T + alpha~) v on the active rows
  auto matvec = [&](const std::vector<T>& v, std::vector<T>& y) {
    for (int i = 0; i < N; ++i) U[i] = V3<T>{T(0.0), T(0.0), T(0.0)};
    apply_rows(N, R, w, v, U);  // U = M^-1 J^T v
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < NK; ++k) {
        const int j = i * NK + k;
        y[j] = T(0.0);
        if (!act[j]) continue;
        T a = alpha_tilde(S, C, k) * v[j];
        for (int l = 0; l < row_nodes(k); ++l) a += dot(R.G(i, k, l), U[row_node(i, k, l)]);
        y[j] = a;
      }
  };
  int mv = 0;
  for (;;) {
    eval_rows(S, C, X, XS, theta, R);
    r_end = residual(S, C, R, w, lam, XS);
    if (r_end <= C.tol || mv >= C.iters) break;
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < NK; ++k) {
        const int j = i * NK + k;
        act[j] = (k <= R_PITCH && R.ON(i, k) && val(row_wgrad2(R, w, i, k)) != 0.0) ? 1 : 0;
        if (!act[j]) { D[j] = T(1.0); b[j] = T(0.0); continue; }
        const T at = alpha_tilde(S, C, k);
        D[j] = row_wgrad2(R, w, i, k) + at;
        b[j] = -(R.C(i, k) + at * lam[j]);
      }
    // PCR from dlambda = 0: z = D^-1 r, p = z, q = A p
    for (int j = 0; j < n; ++j) { x[j] = T(0.0); z[j] = act[j] ? b[j] / D[j] : T(0.0); p[j] = z[j]; }
    matvec(z, Az);
    ++mv;
    for (int j = 0; j < n; ++j) q[j] = Az[j];
    T zaz = dot_act(z, Az);
    for (int it = 0; it < C.pcr_iters && mv < C.iters; ++it) {
      T qs(0.0);
      for (int j = 0; j < n; ++j) if (act[j]) qs += q[j] * q[j] / D[j];
      if (!(val(qs) > 0.0)) break;
      const T alpha = zaz / qs;
      for (int j = 0; j < n; ++j) {
        if (!act[j]) continue;
        x[j] += alpha * p[j];
        z[j] -= alpha * q[j] / D[j];
      }
      matvec(z, Az);
      ++mv;
      const T zaz_new = dot_act(z, Az);
      const T beta = zaz_new / zaz;
      zaz = zaz_new;
      for (int j = 0; j < n; ++j) {
        if (!act[j]) continue;
        p[j] = z[j] + beta * p[j];
        q[j] = Az[j] + beta * q[j];
      }
    }
    for (int j = 0; j < n; ++j) if (act[j]) lam[j] += x[j];
    apply_rows(N, R, w, x, X);  // x += M^-1 J^T dlambda at the linearisation point
  }
  return mv;
}

// ---------------------------------------------------------------- warm-start network
// The learned warm start reads 24 features per constraint row at the predicted positions
// of a substep and predicts the row's multiplier over m g h^2.  Row frame: horizontal
// unit tangent t (stretch: the row's segment; bend: the segment into node i; contact:
// the segment out of node i, the one into it at the last node; friction x / y: world
// x / y), b = z x t, z.  Features: one-hot row kind (6); height of the row's first node
// above its contact height, / L0 (1); second and third node relative to the first, in
// the frame, / L0 (6); velocities of the nodes in the frame, times h / L0 (9); rest angle
// of a yaw row (1); the row's multiplier of the previous substep / (m g h^2) (1).
constexpr int kFeat = 24, kHid = 128;
constexpr int kMlpParams = kHid * kFeat + kHid + kHid * kHid + kHid + kHid + 1;

// Round to the nearest bfloat16 (ties to even), the operand precision of the network.
double bf16r(double a) {
  float f = (float)a;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

double silu_exact(double z) { return z / (1.0 + std::exp(-z)); }

// One forward pass: operands (features, W1, W2, first hidden layer) rounded to bfloat16
// as the tensor cores read them, everything else in FP64.
double mlp_forward(const double* P, const double* f) {
  const double* W1 = P;
  const double* b1 = W1 + kHid * kFeat;
  const double* W2 = b1 + kHid;
  const double* b2 = W2 + kHid * kHid;
  const double* w3 = b2 + kHid;
  const double b3 = w3[kHid];
  double h1[kHid];
  for (int o = 0; o < kHid; ++o) {
    double z = b1[o];
    for (int i = 0; i < kFeat; ++i) z += bf16r(W1[o * kFeat + i]) * bf16r(f[i]);
    h1[o] = bf16r(silu_exact(z));
  }
  double y = b3;
  for (int o = 0; o < kHid; ++o) {
    double z = b2[o];
    for (int i = 0; i < kHid; ++i) z += bf16r(W2[o * kHid + i]) * h1[i];
    y += w3[o] * silu_exact(z);
  }
  return y;
}

// Features of every row of one snake ([N][6][24]) at positions X, velocities v,
// previous multipliers lam and rest angles theta.
template <class T>
void row_features(const Snake<T>& S, const Cfg& C, const std::vector<V3<T>>& X, const V3<T>* v,
                  const std::vector<T>& lam, const std::vector<T>& theta, double* F) {
  const int N = S.N;
  const double L0 = val(S.L0), h = C.h;
  const double lsc = 1.0 / (val(S.mass) * 9.81 * h * h);
  auto P = [&](int i) { return V3<double>{val(X[i].x), val(X[i].y), val(X[i].z)}; };
  auto dirh = [&](int b, int a, double& tx, double& ty) {
    double ex = val(X[b].x) - val(X[a].x), ey = val(X[b].y) - val(X[a].y);
    double n = std::sqrt(ex * ex + ey * ey);
    if (n > 0.0) { tx = ex / n; ty = ey / n; } else { tx = 1.0; ty = 0.0; }
  };
  for (int i = 0; i < N; ++i) {
    for (int k = 0; k < NK; ++k) {
      double* f = F + ((size_t)i * NK + k) * kFeat;
      for (int c = 0; c < kFeat; ++c) f[c] = 0.0;
      bool ex = (k == R_STRETCH) ? (i <= N - 2)
              : (k == R_YAW || k == R_PITCH) ? (i >= 1 && i <= N - 2)
              : (C.contact && i >= S.nfix);
      if (!ex) continue;
      f[k] = 1.0;
      int a, b = -1, c = -1;
      double tx, ty;
      if (k == R_STRETCH) { a = i; b = i + 1; dirh(i + 1, i, tx, ty); }
      else if (k == R_YAW || k == R_PITCH) { a = i - 1; b = i; c = i + 1; dirh(i, i - 1, tx, ty); }
      else {
        a = i;
        if (k == R_CONTACT) { if (i + 1 <= N - 1) dirh(i + 1, i, tx, ty); else dirh(i, i - 1, tx, ty); }
        else if (k == R_FX) { tx = 1.0; ty = 0.0; }
        else { tx = 0.0; ty = 1.0; }
      }
      V3<double> pa = P(a);
      f[6] = (pa.z - val(S.radius)) / L0;
      int nodes[3] = {a, b, c};
      for (int u = 1; u < 3; ++u) {
        if (nodes[u] < 0) continue;
        V3<double> d = sub(P(nodes[u]), pa);
        f[7 + 3 * (u - 1)] = (d.x * tx + d.y * ty) / L0;
        f[8 + 3 * (u - 1)] = (-d.x * ty + d.y * tx) / L0;
        f[9 + 3 * (u - 1)] = d.z / L0;
      }
      for (int u = 0; u < 3; ++u) {
        if (nodes[u] < 0) continue;
        const V3<T>& vv = v[nodes[u]];
        f[13 + 3 * u] = (val(vv.x) * tx + val(vv.y) * ty) * h / L0;
        f[14 + 3 * u] = (-val(vv.x) * ty + val(vv.y) * tx) * h / L0;
        f[15 + 3 * u] = val(vv.z) * h / L0;
      }
      if (k == R_YAW) f[22] = val(theta[i]);
      f[23] = val(lam[i * NK + k]) * lsc;
    }
  }
}

// ---------------------------------------------------------------- one env-step
// Advances one snake by one env-step of n_sub substeps.  Returns the max residual over
// the substeps and adds the number of Jacobi updates to *iters.
template <class T>
double snake_step(const Snake<T>& S, const Cfg& C, long long step_index, V3<T>* x,
                  V3<T>* v, T* press, T* lam_io, const double* ucmd, int* iters,
                  const double* mlp /* network parameters for warm = 2, or null */,
                  double* feat0 = nullptr /* if set: features of substep 0, then return */) {
  const int N = S.N;
  const double h = C.h;
  std::vector<double> w(N);
  for (int i = 0; i < N; ++i) w[i] = (i < S.nfix) ? 0.0 : 1.0 / val(S.mass);
  std::vector<V3<T>> X(x, x + N), XS(N);
  std::vector<T> lam(lam_io, lam_io + (size_t)N * NK), lnew((size_t)N * NK), dl((size_t)N * NK);
  std::vector<T> theta(N, T(0.0));
  Rows<T> R; R.init(N);
  double rmax = 0.0;
  for (int s = 0; s < C.n_sub; ++s) {
    // (a1) gait target, sampled at the end of the substep (Eq. 11 uses a(t + h)).
    double tnext = ((double)step_index * C.n_sub + s + 1) * h;
    // (a2) antagonistic chambers (Sec. III): a > 0 inflates the right chamber, a < 0 the
    // left; each chamber follows its target through a first-order latency,
    // p <- p^ + (p - p^) exp(-h / tau), tau = tau_inflate when rising else tau_deflate.
    // With the chamber law of Sec. V-A instead (C.latency == 1) the chambers move once
    // per law step of C.law_every substeps, towards the target at the end of that step,
    // and hold their value in between.
    const long long g = step_index * C.n_sub + s;
    const bool law_now = C.latency == 1 && g % C.law_every == 0;
    const double tlaw = (double)(g + C.law_every) * h;
    for (int k = 0; k < S.L && (C.latency == 0 || law_now); ++k) {
      double a = ucmd ? ucmd[k] : gait_target(S, k, C.latency == 0 ? tnext : tlaw);
      double tgt[2] = {std::max(a, 0.0), std::max(-a, 0.0)};
      for (int ch = 0; ch < 2; ++ch) {
        T& p = press[2 * k + ch];
        if (C.latency == 1) { p = chamber_law(p, tgt[ch], C); continue; }
        T tau = (tgt[ch] > val(p)) ? S.tau_inf : S.tau_def;
        p = tgt[ch] + (p - tgt[ch]) * exp(T(-h) / tau);
      }
    }
    // (a3) rest angle of bend rows inside link k: theta = G (p_R - p_L) L0 (Eq. 3-4 with
    // an inextensible centre layer); straight (0) at the rigid connector nodes.
    for (int i = 1; i <= N - 2; ++i) {
      if (i % S.seg == 0) { theta[i] = T(0.0); continue; }
      int k = i / S.seg;
      theta[i] = S.gain * (press[2 * k] - press[2 * k + 1]) * S.L0;
    }
    // (a4) predict with gravity (first-order implicit Euler, Sec. IV-D).
    for (int i = 0; i < N; ++i) {
      XS[i] = X[i];
      if (w[i] > 0.0) {
        v[i].x += h * C.g[0]; v[i].y += h * C.g[1]; v[i].z += h * C.g[2];
        X[i].x = X[i].x + h * v[i].x; X[i].y = X[i].y + h * v[i].y; X[i].z = X[i].z + h * v[i].z;
      }
    }
    if (feat0) { row_features(S, C, X, v, lam, theta, feat0); return 0.0; }
    // multipliers: cold (0), beta x the previous substep's values, or in the learned mode
    // at the substeps s with s % net_every == 0, on the row kinds the network predicts
    // (every kind, the bilateral kinds or the stretch rows), beta_net x the previous value
    // plus the network's prediction.  A non-zero start also moves the nodes by
    // M^-1 J^T lambda0 (gradients at the predicted positions), so that
    // M (x - x~) = J^T lambda holds from the first iterate on.
    if (C.warm == 0) for (auto& l : lam) l = T(0.0);
    else {
      std::vector<double> y(lam.size(), 0.0);
      std::vector<char> pred(lam.size(), 0);
      if (C.warm == 2 && mlp && s % C.net_every == 0) {
        std::vector<double> F((size_t)N * NK * kFeat);
        row_features(S, C, X, v, lam, theta, F.data());
        for (size_t j = 0; j < lam.size(); ++j)
          if (C.net_rows == 0 || (int)(j % NK) <= (C.net_rows == 1 ? R_PITCH : R_STRETCH)) {
            pred[j] = 1;
            y[j] = mlp_forward(mlp, &F[j * kFeat]);
          }
      }
      const double sc = val(S.mass) * 9.81 * h * h;
      for (size_t j = 0; j < lam.size(); ++j)
        lam[j] = (pred[j] ? C.beta_net : C.beta) * lam[j] + T(y[j] * sc);
    }
    if (C.warm != 0) {
      eval_rows(S, C, X, XS, theta, R);
      for (int i = 0; i < N; ++i)
        for (int kk = 0; kk < NK; ++kk) {
          int j = i * NK + kk;
          dl[j] = (R.ON(i, kk) && val(row_wgrad2(R, w, i, kk)) != 0.0) ? lam[j] : T(0.0);
          lam[j] = dl[j];
        }
      apply_rows(N, R, w, dl, X);
    }
    if (C.solver == 1) {  // Newton + PCR instead of the Jacobi relaxation
      double r = 0.0;
      *iters += newton_pcr(S, C, X, XS, theta, R, w, lam, r);
      rmax = std::max(rmax, r);
    }
    // (a5/a6) Jacobi iterations.
    int k = 0;
    for (; C.solver == 0; ++k) {
      eval_rows(S, C, X, XS, theta, R);
      double r = residual(S, C, R, w, lam, XS);
      if (r <= C.tol || k >= C.iters) { rmax = std::max(rmax, r); break; }
      // new multipliers from (x^k, lambda^k) only
      for (int i = 0; i < N; ++i) {
        for (int kk = 0; kk < NK; ++kk) {
          int j = i * NK + kk;
          lnew[j] = lam[j];
          if (!R.ON(i, kk)) continue;
          T wg = row_wgrad2(R, w, i, kk);
          if (val(wg) == 0.0) continue;
          if (kk == R_STRETCH || kk == R_YAW || kk == R_PITCH) {
            T at = alpha_tilde(S, C, kk);
            T dlam = (-R.C(i, kk) - at * lam[j]) / (wg + at);
            lnew[j] = lam[j] + C.omega * dlam;
          } else if (kk == R_CONTACT) {
            T dlam = -R.C(i, kk) / wg;
            lnew[j] = tmax(T(0.0), lam[j] + C.omega * dlam);      // lambda_n >= 0 (Eq. 7)
          }
        }
        if (R.ON(i, R_FX) && w[i] > 0.0) {
          // friction pair projected onto the disc |lambda_t| <= mu lambda_n, with
          // lambda_n of the current iterate (Jacobi)
          int jx = i * NK + R_FX, jy = i * NK + R_FY;
          T tx = lam[jx] + C.omega * (-R.C(i, R_FX) / w[i]);
          T ty = lam[jy] + C.omega * (-R.C(i, R_FY) / w[i]);
          if (S.mu_side > 0.0) {  // ellipse of the body frame
            double bx, by;
            body_tangent(XS, N, i, bx, by);
            project_ellipse(tx, ty, bx, by, val(S.mu), S.mu_side, lam[i * NK + R_CONTACT]);
          } else {
            T rad = S.mu * lam[i * NK + R_CONTACT];
            double n2 = val(tx) * val(tx) + val(ty) * val(ty);
            if (n2 > val(rad) * val(rad)) {
              if (val(rad) <= 0.0) { tx = T(0.0); ty = T(0.0); }
              else { T nrm = sqrt(tx * tx + ty * ty); tx = tx * rad / nrm; ty = ty * rad / nrm; }
            }
          }
          lnew[jx] = tx; lnew[jy] = ty;
        }
      }
      for (size_t j = 0; j < lam.size(); ++j) { dl[j] = lnew[j] - lam[j]; lam[j] = lnew[j]; }
      apply_rows(N, R, w, dl, X);
    }
    if (C.solver == 0) *iters += k;
    // (a7) velocity from the substep displacement, exponential damping d [1/s].
    T damp = exp(-S.damp * h);
    for (int i = 0; i < N; ++i) {
      if (w[i] == 0.0) { v[i] = V3<T>{T(0.0), T(0.0), T(0.0)}; continue; }
      v[i] = scl(sub(X[i], XS[i]), damp / h);
    }
  }
  for (int i = 0; i < N; ++i) x[i] = X[i];
  for (size_t j = 0; j < lam.size(); ++j) lam_io[j] = lam[j];
  return rmax;
}

struct Offsets {
  std::vector<long long> node, link;
};
Offsets offsets(int n, const int* nl, const int* seg) {
  Offsets o; o.node.resize(n + 1); o.link.resize(n + 1);
  o.node[0] = o.link[0] = 0;
  for (int s = 0; s < n; ++s) { o.node[s + 1] = o.node[s] + (long long)nl[s] * seg[s] + 1; o.link[s + 1] = o.link[s] + nl[s]; }
  return o;
}

}  // namespace

extern "C" {

int oracle_nprm() { return NPRM; }
int oracle_mlp_params() { return kMlpParams; }
int oracle_ncfg() { return NCFG; }

// Straight initial pose along the heading yaw0 from (x0, y0, z0), at rest, chambers
// empty, multipliers zero.
int oracle_init(int n, const int* nl, const int* seg, const double* prm, double* x, double* v,
                double* press, double* lam) {
  Offsets o = offsets(n, nl, seg);
  for (int s = 0; s < n; ++s) {
    const double* p = prm + (size_t)s * NPRM;
    double c = std::cos(p[P_YAW0]), sn = std::sin(p[P_YAW0]);
    for (long long i = o.node[s]; i < o.node[s + 1]; ++i) {
      double d = (double)(i - o.node[s]) * p[P_L0];
      x[3 * i] = p[P_X0] + d * c; x[3 * i + 1] = p[P_Y0] + d * sn; x[3 * i + 2] = p[P_Z0];
      v[3 * i] = v[3 * i + 1] = v[3 * i + 2] = 0.0;
      for (int k = 0; k < NK; ++k) lam[i * NK + k] = 0.0;
    }
    for (long long k = o.link[s]; k < o.link[s + 1]; ++k) press[2 * k] = press[2 * k + 1] = 0.0;
  }
  return 0;
}

// Advances every snake by n_steps env-steps.  x, v: [nodes][3]; press: [links][2];
// lam: [nodes][6]; ucmd: optional [links] command held for these steps (null = gait);
// resid/iters: per snake, max residual and total updates of the last step;
// tip: optional [n_steps][n][3] last-node positions after each step;
// mlp: network parameters (19841 doubles) used when the configuration's warm = 2.
int oracle_step(int n, const int* nl, const int* seg, const int* nfix, const double* prm,
                const double* cfg, long long step_index, int n_steps, double* x, double* v,
                double* press, double* lam, const double* ucmd, double* resid, int* iters,
                double* tip, const double* mlp, int n_threads) {
  Cfg C = load_cfg(cfg);
  Offsets o = offsets(n, nl, seg);
  long long total_nodes = o.node[n];
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int s = 0; s < n; ++s) {
    Snake<double> S = load_snake<double>(nl, seg, nfix, prm, s);
    V3<double>* xs = reinterpret_cast<V3<double>*>(x + 3 * o.node[s]);
    V3<double>* vs = reinterpret_cast<V3<double>*>(v + 3 * o.node[s]);
    double* ps = press + 2 * o.link[s];
    double* ls = lam + NK * o.node[s];
    const double* us = ucmd ? ucmd + o.link[s] : nullptr;
    double r = 0.0;
    for (int st = 0; st < n_steps; ++st) {
      int it = 0;
      r = snake_step(S, C, step_index + st, xs, vs, ps, ls, us, &it, mlp);
      if (iters) iters[s] = it;
      if (tip) {
        const V3<double>& t = xs[S.N - 1];
        double* d = tip + ((size_t)st * n + s) * 3;
        d[0] = t.x; d[1] = t.y; d[2] = t.z;
      }
    }
    if (resid) resid[s] = r;
  }
  return 0;
}

// Features [nodes][6][24] of every row at the predicted state of substep 0 of env-step
// step_index, from the current state (which is not modified).
int oracle_features(int n, const int* nl, const int* seg, const int* nfix, const double* prm,
                    const double* cfg, long long step_index, const double* x, const double* v,
                    const double* press, const double* lam, const double* ucmd, double* feat) {
  Cfg C = load_cfg(cfg);
  Offsets o = offsets(n, nl, seg);
  for (int s = 0; s < n; ++s) {
    Snake<double> S = load_snake<double>(nl, seg, nfix, prm, s);
    std::vector<V3<double>> X(S.N), V(S.N);
    for (int i = 0; i < S.N; ++i) {
      long long g = o.node[s] + i;
      X[i] = {x[3 * g], x[3 * g + 1], x[3 * g + 2]};
      V[i] = {v[3 * g], v[3 * g + 1], v[3 * g + 2]};
    }
    std::vector<double> P(press + 2 * o.link[s], press + 2 * o.link[s + 1]);
    std::vector<double> Lm(lam + NK * o.node[s], lam + NK * o.node[s + 1]);
    int it = 0;
    snake_step(S, C, step_index, X.data(), V.data(), P.data(), Lm.data(),
               ucmd ? ucmd + o.link[s] : nullptr, &it, nullptr, feat + (size_t)o.node[s] * NK * kFeat);
  }
  return 0;
}

// Network outputs y[rows] for features [rows][24].
int oracle_mlp_forward(const double* params, long long rows, const double* feat, double* y) {
  for (long long r = 0; r < rows; ++r) y[r] = mlp_forward(params, feat + r * kFeat);
  return 0;
}

// Row values c[N][6], existence on[N][6] and node gradients g[N][6][3 local][3] of one
// snake at positions x (with substep-start positions xs for the friction rows) and
// chamber pressures press (which set the yaw rest angles).
int oracle_rows(int nl, int seg, const double* prm1, const double* cfg, const double* x,
                const double* xs, const double* press, double* c, double* g, int* on) {
  int one_nl = nl, one_seg = seg, zero = 0;
  Snake<double> S = load_snake<double>(&one_nl, &one_seg, &zero, prm1, 0);
  Cfg C = load_cfg(cfg);
  std::vector<V3<double>> X(S.N), XS(S.N);
  for (int i = 0; i < S.N; ++i) { X[i] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]}; XS[i] = {xs[3 * i], xs[3 * i + 1], xs[3 * i + 2]}; }
  std::vector<double> theta(S.N, 0.0);
  for (int i = 1; i <= S.N - 2; ++i) {
    if (i % S.seg == 0) continue;
    int k = i / S.seg;
    theta[i] = S.gain * (press[2 * k] - press[2 * k + 1]) * S.L0;
  }
  Rows<double> R; R.init(S.N);
  eval_rows(S, C, X, XS, theta, R);
  for (int i = 0; i < S.N * NK; ++i) { c[i] = R.c[i]; on[i] = R.on[i]; }
  for (int i = 0; i < S.N * NK * 3; ++i) { g[3 * i] = R.g[i].x; g[3 * i + 1] = R.g[i].y; g[3 * i + 2] = R.g[i].z; }
  return 0;
}

// The normalised residual residual() reports for one snake (n_fixed leading nodes held)
// at positions x, substep-start positions xs, chamber pressures press and multipliers
// lam[N][6]: the value the Jacobi and Newton loops compare against the tolerance.
double oracle_residual(int nl, int seg, int nfix, const double* prm1, const double* cfg,
                       const double* x, const double* xs, const double* press, const double* lam) {
  int one_nl = nl, one_seg = seg, one_fix = nfix;
  Snake<double> S = load_snake<double>(&one_nl, &one_seg, &one_fix, prm1, 0);
  Cfg C = load_cfg(cfg);
  std::vector<V3<double>> X(S.N), XS(S.N);
  for (int i = 0; i < S.N; ++i) { X[i] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]}; XS[i] = {xs[3 * i], xs[3 * i + 1], xs[3 * i + 2]}; }
  std::vector<double> theta(S.N, 0.0), w(S.N), L(lam, lam + (size_t)S.N * NK);
  for (int i = 1; i <= S.N - 2; ++i) {
    if (i % S.seg == 0) continue;
    int k = i / S.seg;
    theta[i] = S.gain * (press[2 * k] - press[2 * k + 1]) * S.L0;
  }
  for (int i = 0; i < S.N; ++i) w[i] = (i < S.nfix) ? 0.0 : 1.0 / S.mass;
  Rows<double> R; R.init(S.N);
  eval_rows(S, C, X, XS, theta, R);
  return residual(S, C, R, w, L, XS);
}

// Forward-mode gradient of the calibration loss
//   L_s = (1/n_steps) sum_t |tip_s(t) - target_s(t)|^2
// with respect to (alpha_b, damping, tau_inflate, tau_deflate, gain) of each snake,
// starting from the given state (not modified).  loss: [n]; grad: [n][5].
int oracle_calib_grad(int n, const int* nl, const int* seg, const int* nfix, const double* prm,
                      const double* cfg, long long step_index, int n_steps, const double* x0,
                      const double* v0, const double* p0, const double* lam0,
                      const double* target, double* loss, double* grad, int n_threads) {
  typedef Dual<5> D;
  Cfg C = load_cfg(cfg);
  Offsets o = offsets(n, nl, seg);
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
  for (int s = 0; s < n; ++s) {
    Snake<D> S = load_snake<D>(nl, seg, nfix, prm, s);
    S.alpha_b.d[0] = 1.0; S.damp.d[1] = 1.0; S.tau_inf.d[2] = 1.0; S.tau_def.d[3] = 1.0; S.gain.d[4] = 1.0;
    std::vector<V3<D>> X(S.N), V(S.N);
    for (int i = 0; i < S.N; ++i) {
      long long g = o.node[s] + i;
      X[i] = {D(x0[3 * g]), D(x0[3 * g + 1]), D(x0[3 * g + 2])};
      V[i] = {D(v0[3 * g]), D(v0[3 * g + 1]), D(v0[3 * g + 2])};
    }
    std::vector<D> P(2 * S.L), Lm((size_t)S.N * NK);
    for (int k = 0; k < 2 * S.L; ++k) P[k] = D(p0[2 * o.link[s] + k]);
    for (int j = 0; j < S.N * NK; ++j) Lm[j] = D(lam0[NK * o.node[s] + j]);
    D acc(0.0);
    for (int st = 0; st < n_steps; ++st) {
      int it = 0;
      snake_step(S, C, step_index + st, X.data(), V.data(), P.data(), Lm.data(), nullptr, &it, nullptr);
      const double* tg = target + ((size_t)st * n + s) * 3;
      V3<D> d{X[S.N - 1].x - tg[0], X[S.N - 1].y - tg[1], X[S.N - 1].z - tg[2]};
      acc += dot(d, d);
    }
    acc = acc / (double)n_steps;
    loss[s] = acc.v;
    for (int k = 0; k < 5; ++k) grad[5 * s + k] = acc.d[k];
  }
  return 0;
}

}  // extern "C"
