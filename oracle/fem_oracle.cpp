// FP64 CPU oracle of the tetrahedral soft link (test infrastructure).
//
// Only the tests, the smoke check and the CPU leg of the benchmark use this file.  It is
// independent of the CUDA path: it shares no kernels, headers or helpers with it.
//
// What it computes, per link of a batch that shares one mesh, per substep of a frame:
//  - chamber pressure from the open-loop command of Eq. 9 sampled at t + h (amplitude in
//    Pa, signed: > 0 drives the right chamber, < 0 the left one);
//  - actuation rows (Sec. III-A, Eq. 1-2): distance rows along the active chamber with
//    rest length r eps(p), eps(p) = 1 + |p| / Y; only the expanding chamber's rows exist;
//  - distance rows of constant rest length for the inextensible centre layer and the
//    fibre-held perimeter (Sec. V), each with its own compliance;
//  - tetrahedral finite elements (Sec. III-B, Eq. 5): per tetrahedron the six corotational
//    strains in Voigt order [xx yy zz yz xz xy] (tensor shears) of F = R S, c = S - I,
//    with the element compliance E = C / (V Y) of the printed 6x6 matrix C (1, -nu on the
//    normal block; 1 + nu on the shear diagonal);
//  - lumped masses (Sec. IV-A): each particle a quarter of every adjacent element's mass;
//  - implicit prediction and the Newton + preconditioned conjugate residual solve of
//    Sec. IV-D on the Schur system of Eq. 8, (J M^-1 J^T + E / h^2) dlambda =
//    -(c + E lambda / h^2), diagonal (Jacobi) preconditioner, multipliers from 0 at every
//    substep;
//  - velocity v = (x - x_s) / h damped by exp(-d h).
// Readings: the gradient of a strain row holds R fixed (corotational linearisation), so
// d c / d x_a = R Sigma_k g_a with g_a the shape-function gradient of vertex a and Sigma_k
// the symmetric unit tensor of Voigt entry k; the polar factor is taken from the
// eigen-decomposition of F^T F (cyclic Jacobi rotations), which needs det F > 0.
//
// Pinned by tests/test_fem_oracle_pins.py: the polar factor against scipy's polar
// decomposition; strains of rigid motions (zero), of stretches (exact) and of shears;
// gradients against central differences at rotated rest states; the static solution of
// a lightly loaded link against the textbook linear FEM stiffness K u = f assembled
// independently from shape functions (with and without compliant distance rows); the
// actuation rest length of Eq. 2; linear momentum conservation; rest invariance.
// Parity unpinned: frames at the paper's fixed budget stop far from convergence and have
// no closed form; the stepping function is pinned through its converged limits and its
// invariants, and the GPU path is checked against it.
#include <omp.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

constexpr int kNF = 11;  // per-link parameters
enum { Y_, NU_, RHO_, DAMP_, A_INEXT_, A_PERIM_, A_ACT_, P_AMP_, P_FREQ_, P_PHASE_, P_OFF_ };
constexpr int kNC = 8;   // config: dt, n_sub, iters, tol, pcr_iters, gravity (3)
enum { KIND_INEXT = 0, KIND_PERIM = 1, KIND_LEFT = 2, KIND_RIGHT = 3 };

template <class T>
struct V3 {
  T x, y, z;
};
template <class T> V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

template <class T>
struct M3 {
  T m[3][3];
};

template <class T>
M3<T> mul(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = 0;
      for (int k = 0; k < 3; ++k) s += A.m[i][k] * B.m[k][j];
      C.m[i][j] = s;
    }
  return C;
}

template <class T>
M3<T> transpose(const M3<T>& A) {
  M3<T> B;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B.m[i][j] = A.m[j][i];
  return B;
}

template <class T>
T det(const M3<T>& A) {
  return A.m[0][0] * (A.m[1][1] * A.m[2][2] - A.m[1][2] * A.m[2][1]) -
         A.m[0][1] * (A.m[1][0] * A.m[2][2] - A.m[1][2] * A.m[2][0]) +
         A.m[0][2] * (A.m[1][0] * A.m[2][1] - A.m[1][1] * A.m[2][0]);
}

template <class T>
M3<T> inverse(const M3<T>& A) {
  const T d = det(A);
  M3<T> B;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // cofactor of A[j][i]
      const int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
      B.m[i][j] = (A.m[r0][c0] * A.m[r1][c1] - A.m[r0][c1] * A.m[r1][c0]) / d;
    }
  return B;
}

// Symmetric eigen-decomposition A = Q diag(w) Q^T by cyclic Jacobi rotations.
template <class T>
void sym_eig(M3<T> A, M3<T>& Q, T w[3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Q.m[i][j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    const T off = A.m[0][1] * A.m[0][1] + A.m[0][2] * A.m[0][2] + A.m[1][2] * A.m[1][2];
    const T diag = A.m[0][0] * A.m[0][0] + A.m[1][1] * A.m[1][1] + A.m[2][2] * A.m[2][2];
    if (off <= T(1e-300) || off <= diag * T(sizeof(T) == 8 ? 1e-32 : 1e-16)) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A.m[p][q] == T(0)) continue;
        // rotation angle that zeroes A[p][q]
        const T theta = (A.m[q][q] - A.m[p][p]) / (T(2) * A.m[p][q]);
        const T t = (theta >= 0 ? T(1) : T(-1)) / (std::fabs(theta) + std::sqrt(theta * theta + T(1)));
        const T c = T(1) / std::sqrt(t * t + T(1)), s = t * c;
        for (int k = 0; k < 3; ++k) {  // A <- A G (columns p, q)
          const T akp = A.m[k][p], akq = A.m[k][q];
          A.m[k][p] = c * akp - s * akq;
          A.m[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // A <- G^T A (rows p, q)
          const T apk = A.m[p][k], aqk = A.m[q][k];
          A.m[p][k] = c * apk - s * aqk;
          A.m[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {  // Q <- Q G
          const T qkp = Q.m[k][p], qkq = Q.m[k][q];
          Q.m[k][p] = c * qkp - s * qkq;
          Q.m[k][q] = s * qkp + c * qkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) w[i] = A.m[i][i];
}

// Polar decomposition F = R S with S = (F^T F)^(1/2) symmetric positive definite and
// R = F S^-1 (a rotation when det F > 0).  NaN when det F <= 0.
template <class T>
void polar(const M3<T>& F, M3<T>& R, M3<T>& S) {
  const T nan = std::numeric_limits<T>::quiet_NaN();
  if (!(det(F) > T(0))) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) R.m[i][j] = S.m[i][j] = nan;
    return;
  }
  M3<T> Q;
  T w[3];
  sym_eig(mul(transpose(F), F), Q, w);
  M3<T> Si;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = 0, si = 0;
      for (int k = 0; k < 3; ++k) {
        const T sk = std::sqrt(w[k]);
        s += Q.m[i][k] * sk * Q.m[j][k];
        si += Q.m[i][k] / sk * Q.m[j][k];
      }
      S.m[i][j] = s;
      Si.m[i][j] = si;
    }
  R = mul(F, Si);
}

// Symmetric unit tensor of Voigt entry k (tensor shears: entry yz is the tensor's (1,2)
// and (2,1) components, each 1/2, so that sum_ij Sigma_ij eps_ij = eps_k).
template <class T>
M3<T> voigt_unit(int k) {
  M3<T> E{};
  static const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
  if (k < 3) {
    E.m[k][k] = T(1);
  } else {
    E.m[I[k]][J[k]] = T(0.5);
    E.m[J[k]][I[k]] = T(0.5);
  }
  return E;
}

template <class T>
V3<T> matvec(const M3<T>& A, V3<T> v) {
  return {A.m[0][0] * v.x + A.m[0][1] * v.y + A.m[0][2] * v.z,
          A.m[1][0] * v.x + A.m[1][1] * v.y + A.m[1][2] * v.z,
          A.m[2][0] * v.x + A.m[2][1] * v.y + A.m[2][2] * v.z};
}

// Rest data of one element: shape-function gradients g_a (F = sum_a x_a g_a^T) and volume.
template <class T>
struct TetRest {
  V3<T> g[4];
  T vol;
};

template <class T>
TetRest<T> tet_rest(const V3<T> X[4]) {
  M3<T> Dm;
  for (int a = 0; a < 3; ++a) {
    const V3<T> e = X[a + 1] - X[0];
    Dm.m[0][a] = e.x;
    Dm.m[1][a] = e.y;
    Dm.m[2][a] = e.z;
  }
  const M3<T> B = inverse(Dm);  // F = Ds B: row a of B multiplies (x_{a+1} - x_0)
  TetRest<T> r;
  r.g[0] = V3<T>{0, 0, 0};
  for (int a = 0; a < 3; ++a) {
    r.g[a + 1] = V3<T>{B.m[a][0], B.m[a][1], B.m[a][2]};
    r.g[0] = r.g[0] - r.g[a + 1];
  }
  r.vol = det(Dm) / T(6);
  return r;
}

// Corotational strain of one element at positions x, with the gradient of each strain
// row with respect to each vertex (R held fixed) and the polar rotation.
template <class T>
void tet_strain(const V3<T> x[4], const TetRest<T>& tr, T c[6], V3<T> G[6][4], M3<T>& R) {
  M3<T> F{};
  for (int a = 1; a < 4; ++a) {
    const V3<T> d = x[a] - x[0];
    const T dv[3] = {d.x, d.y, d.z};
    const T gv[3] = {tr.g[a].x, tr.g[a].y, tr.g[a].z};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) F.m[i][j] += dv[i] * gv[j];
  }
  M3<T> S;
  polar(F, R, S);
  const M3<T> RtF = mul(transpose(R), F);
  const T s[3][3] = {{RtF.m[0][0], T(0.5) * (RtF.m[0][1] + RtF.m[1][0]), T(0.5) * (RtF.m[0][2] + RtF.m[2][0])},
                     {0, RtF.m[1][1], T(0.5) * (RtF.m[1][2] + RtF.m[2][1])},
                     {0, 0, RtF.m[2][2]}};
  c[0] = s[0][0] - T(1);
  c[1] = s[1][1] - T(1);
  c[2] = s[2][2] - T(1);
  c[3] = s[1][2];
  c[4] = s[0][2];
  c[5] = s[0][1];
  for (int k = 0; k < 6; ++k) {
    const M3<T> E = voigt_unit<T>(k);
    for (int a = 0; a < 4; ++a) G[k][a] = matvec(R, matvec(E, tr.g[a]));
  }
}

// (C v)_k of the printed compliance pattern: normal block 1 / -nu, shear diagonal 1 + nu.
template <class T>
void compliance_apply(T nu, const T v[6], T out[6]) {
  out[0] = v[0] - nu * (v[1] + v[2]);
  out[1] = v[1] - nu * (v[0] + v[2]);
  out[2] = v[2] - nu * (v[0] + v[1]);
  for (int k = 3; k < 6; ++k) out[k] = (T(1) + nu) * v[k];
}

struct Mesh {
  int P, NT, ND;
  const double* X;
  const int* tets;
  const int* rows;
  const int* kinds;
  const int* fixed;
};

template <class T>
double link_substep(const Mesh& M, const double* prm, const double* cfg, double t_s,
                    const std::vector<TetRest<T>>& TR, const std::vector<T>& w, const std::vector<T>& rest0,
                    std::vector<V3<T>>& x, std::vector<V3<T>>& v, int& mv_out) {
  const int P = M.P, NT = M.NT, ND = M.ND;
  const double dt = cfg[0];
  const int n_sub = (int)cfg[1], cap = (int)cfg[2], pcr_iters = (int)cfg[4];
  const double tol = cfg[3];
  const T h = T(dt / n_sub);
  const V3<T> g{T(cfg[5]), T(cfg[6]), T(cfg[7])};
  const T Y = T(prm[Y_]), nu = T(prm[NU_]);
  // pressure command of Eq. 9 at the end of the substep
  const double tp = t_s + dt / n_sub;
  double u = std::sin(2.0 * M_PI * prm[P_FREQ_] * tp + prm[P_PHASE_]) + prm[P_OFF_];
  u = std::fmin(1.0, std::fmax(-1.0, u));
  const double p = prm[P_AMP_] * u;
  const int active_kind = p > 0.0 ? KIND_RIGHT : (p < 0.0 ? KIND_LEFT : -1);
  const T eps = T(1.0 + std::fabs(p) / prm[Y_]);
  // prediction
  std::vector<V3<T>> xs(P);
  for (int i = 0; i < P; ++i) {
    if (w[i] > T(0)) v[i] = v[i] + h * g;
    xs[i] = x[i];
    if (w[i] > T(0)) x[i] = x[i] + h * v[i];
  }
  // rows: 6 per element, then the distance rows
  const int n = 6 * NT + ND;
  std::vector<T> lam(n, T(0)), D(n, T(1)), b(n, T(0)), dl(n), z(n), pv(n), q(n), Az(n), cval(n), scale(n, T(1));
  std::vector<char> act(n, 0);
  std::vector<V3<T>> Gt((size_t)NT * 24), Gd(ND), U(P);
  std::vector<T> drest(ND), at_d(ND);
  for (int d = 0; d < ND; ++d) {
    const int kind = M.kinds[d];
    const bool on = kind == KIND_INEXT || kind == KIND_PERIM || kind == active_kind;
    act[6 * NT + d] = on ? 1 : 0;
    drest[d] = (kind == KIND_LEFT || kind == KIND_RIGHT) ? rest0[d] * eps : rest0[d];
    const double a = kind == KIND_INEXT ? prm[A_INEXT_] : kind == KIND_PERIM ? prm[A_PERIM_] : prm[A_ACT_];
    at_d[d] = T(a) / (h * h);
    scale[6 * NT + d] = rest0[d];
  }
  const T h2 = h * h;
  // alpha~ v on all rows
  auto alpha_apply = [&](const std::vector<T>& vin, std::vector<T>& out) {
    for (int t = 0; t < NT; ++t) {
      T o[6];
      compliance_apply(nu, &vin[6 * t], o);
      const T s = T(1) / (TR[t].vol * Y * h2);
      for (int k = 0; k < 6; ++k) out[6 * t + k] = s * o[k];
    }
    for (int d = 0; d < ND; ++d) out[6 * NT + d] = at_d[d] * vin[6 * NT + d];
  };
  // U = M^-1 J^T vin over the active rows
  auto apply_jt = [&](const std::vector<T>& vin, std::vector<V3<T>>& out) {
    for (int i = 0; i < P; ++i) out[i] = V3<T>{0, 0, 0};
    for (int t = 0; t < NT; ++t)
      for (int k = 0; k < 6; ++k) {
        const T s = vin[6 * t + k];
        for (int a = 0; a < 4; ++a) {
          const int i = M.tets[4 * t + a];
          out[i] = out[i] + s * Gt[(size_t)t * 24 + k * 4 + a];
        }
      }
    for (int d = 0; d < ND; ++d) {
      if (!act[6 * NT + d]) continue;
      const T s = vin[6 * NT + d];
      out[M.rows[2 * d + 1]] = out[M.rows[2 * d + 1]] + s * Gd[d];
      out[M.rows[2 * d]] = out[M.rows[2 * d]] - s * Gd[d];
    }
    for (int i = 0; i < P; ++i) out[i] = w[i] * out[i];
  };
  auto mat = [&](const std::vector<T>& vin, std::vector<T>& y) {
    apply_jt(vin, U);
    alpha_apply(vin, y);
    for (int t = 0; t < NT; ++t)
      for (int k = 0; k < 6; ++k) {
        T s = y[6 * t + k];
        for (int a = 0; a < 4; ++a) s += dot(Gt[(size_t)t * 24 + k * 4 + a], U[M.tets[4 * t + a]]);
        y[6 * t + k] = s;
      }
    for (int d = 0; d < ND; ++d) {
      const int j = 6 * NT + d;
      if (!act[j]) { y[j] = T(0); continue; }
      y[j] += dot(Gd[d], U[M.rows[2 * d + 1]] - U[M.rows[2 * d]]);
    }
  };
  auto dot_act = [&](const std::vector<T>& a, const std::vector<T>& c) {
    T s = 0;
    for (int j = 0; j < n; ++j) if (act[j]) s += a[j] * c[j];
    return s;
  };
  int mv = 0;
  double r_end = 0.0;
  std::vector<T> al(n);
  for (;;) {
    // linearise at x
    for (int t = 0; t < NT; ++t) {
      V3<T> xt[4];
      for (int a = 0; a < 4; ++a) xt[a] = x[M.tets[4 * t + a]];
      T c[6];
      V3<T> G[6][4];
      M3<T> R;
      tet_strain(xt, TR[t], c, G, R);
      for (int k = 0; k < 6; ++k) {
        cval[6 * t + k] = c[k];
        for (int a = 0; a < 4; ++a) Gt[(size_t)t * 24 + k * 4 + a] = G[k][a];
      }
    }
    for (int d = 0; d < ND; ++d) {
      const V3<T> e = x[M.rows[2 * d + 1]] - x[M.rows[2 * d]];
      const T len = std::sqrt(dot(e, e));
      Gd[d] = (T(1) / len) * e;
      cval[6 * NT + d] = len - drest[d];
    }
    alpha_apply(lam, al);
    double r = 0.0;
    for (int t = 0; t < NT; ++t)
      for (int k = 0; k < 6; ++k) {
        const int j = 6 * t + k;
        T wg = 0;
        for (int a = 0; a < 4; ++a) {
          const V3<T> gg = Gt[(size_t)t * 24 + k * 4 + a];
          wg += w[M.tets[4 * t + a]] * dot(gg, gg);
        }
        T o[6], e6[6] = {0, 0, 0, 0, 0, 0};
        e6[k] = T(1);
        compliance_apply(nu, e6, o);
        D[j] = wg + o[k] / (TR[t].vol * Y * h2);
        act[j] = 1;
      }
    for (int d = 0; d < ND; ++d) {
      const int j = 6 * NT + d;
      if (M.kinds[d] == KIND_LEFT || M.kinds[d] == KIND_RIGHT)
        act[j] = M.kinds[d] == active_kind ? 1 : 0;
      const T wg = w[M.rows[2 * d]] + w[M.rows[2 * d + 1]];
      if (!(wg > T(0))) act[j] = 0;
      D[j] = wg + at_d[d];
    }
    for (int j = 0; j < n; ++j) {
      if (!act[j]) { b[j] = T(0); continue; }
      b[j] = -(cval[j] + al[j]);
      const double rj = std::fabs((double)(cval[j] + al[j])) / (double)scale[j];
      r = std::fmax(r, std::isnan(rj) ? INFINITY : rj);
    }
    r_end = r;
    if (r <= tol || mv >= cap) break;
    for (int j = 0; j < n; ++j) { dl[j] = T(0); z[j] = act[j] ? b[j] / D[j] : T(0); pv[j] = z[j]; }
    mat(z, Az);
    ++mv;
    for (int j = 0; j < n; ++j) q[j] = act[j] ? Az[j] : T(0);
    T zaz = dot_act(z, Az);
    for (int it = 0; it < pcr_iters && mv < cap; ++it) {
      T qs = 0;
      for (int j = 0; j < n; ++j) if (act[j]) qs += q[j] * q[j] / D[j];
      if (!(qs > T(0))) break;
      const T alpha = zaz / qs;
      for (int j = 0; j < n; ++j) {
        if (!act[j]) continue;
        dl[j] += alpha * pv[j];
        z[j] -= alpha * q[j] / D[j];
      }
      mat(z, Az);
      ++mv;
      const T zaz_new = dot_act(z, Az);
      const T beta = zaz_new / zaz;
      zaz = zaz_new;
      for (int j = 0; j < n; ++j) {
        if (!act[j]) continue;
        pv[j] = z[j] + beta * pv[j];
        q[j] = Az[j] + beta * q[j];
      }
    }
    for (int j = 0; j < n; ++j) if (act[j]) lam[j] += dl[j];
    apply_jt(dl, U);
    for (int i = 0; i < P; ++i) x[i] = x[i] + U[i];
  }
  const T damp = T(std::exp(-prm[DAMP_] * (double)h));
  for (int i = 0; i < P; ++i) v[i] = (damp / h) * (x[i] - xs[i]);
  mv_out = mv;
  return r_end;
}

template <class T>
void fem_step_t(int n_links, const Mesh& M, const double* prm, const double* cfg, long long frame,
                int n_frames, double* X, double* Vel, double* resid, int* mv, int n_threads) {
  const int P = M.P;
  // rest data (per link: the density sets the masses)
  std::vector<TetRest<T>> TR(M.NT);
  for (int t = 0; t < M.NT; ++t) {
    V3<T> Xr[4];
    for (int a = 0; a < 4; ++a) {
      const double* p = M.X + 3 * M.tets[4 * t + a];
      Xr[a] = V3<T>{T(p[0]), T(p[1]), T(p[2])};
    }
    TR[t] = tet_rest(Xr);
  }
  std::vector<T> rest0(M.ND);
  for (int d = 0; d < M.ND; ++d) {
    const double* a = M.X + 3 * M.rows[2 * d];
    const double* c = M.X + 3 * M.rows[2 * d + 1];
    rest0[d] = T(std::sqrt((c[0] - a[0]) * (c[0] - a[0]) + (c[1] - a[1]) * (c[1] - a[1]) +
                           (c[2] - a[2]) * (c[2] - a[2])));
  }
  const int n_sub = (int)cfg[1];
  const double h = cfg[0] / n_sub;
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 1)
  for (int l = 0; l < n_links; ++l) {
    const double* pl = prm + (size_t)l * kNF;
    std::vector<T> mass(P, T(0)), w(P, T(0));
    for (int t = 0; t < M.NT; ++t)
      for (int a = 0; a < 4; ++a) mass[M.tets[4 * t + a]] += T(pl[RHO_]) * TR[t].vol / T(4);
    for (int i = 0; i < P; ++i) w[i] = M.fixed[i] ? T(0) : T(1) / mass[i];
    std::vector<V3<T>> x(P), v(P);
    double* xl = X + (size_t)l * P * 3;
    double* vl = Vel + (size_t)l * P * 3;
    for (int i = 0; i < P; ++i) {
      x[i] = V3<T>{T(xl[3 * i]), T(xl[3 * i + 1]), T(xl[3 * i + 2])};
      v[i] = V3<T>{T(vl[3 * i]), T(vl[3 * i + 1]), T(vl[3 * i + 2])};
    }
    double r = 0.0;
    int mv_tot = 0;
    for (int f = 0; f < n_frames; ++f) {
      r = 0.0;  // reported: the largest residual and the products of the last frame
      mv_tot = 0;
      for (int s = 0; s < n_sub; ++s) {
        int mvs = 0;
        const double t_s = (double)((frame + f) * n_sub + s) * h;
        r = std::fmax(r, link_substep<T>(M, pl, cfg, t_s, TR, w, rest0, x, v, mvs));
        mv_tot += mvs;
      }
    }
    for (int i = 0; i < P; ++i) {
      xl[3 * i] = x[i].x; xl[3 * i + 1] = x[i].y; xl[3 * i + 2] = x[i].z;
      vl[3 * i] = v[i].x; vl[3 * i + 1] = v[i].y; vl[3 * i + 2] = v[i].z;
    }
    resid[l] = r;
    mv[l] = mv_tot;
  }
}

}  // namespace

extern "C" {

int fem_oracle_nprm() { return kNF; }
int fem_oracle_ncfg() { return kNC; }

// Polar decomposition of one 3x3 matrix (row-major): F = R S.
void fem_oracle_polar(const double* F, double* R, double* S) {
  M3<double> f, r, s;
  std::memcpy(f.m, F, sizeof(f.m));
  polar(f, r, s);
  std::memcpy(R, r.m, sizeof(r.m));
  std::memcpy(S, s.m, sizeof(s.m));
}

// Strain rows of one element: rest vertices Xr [4][3], current x [4][3] -> c [6],
// gradients G [6][4][3] (R fixed), rotation R [3][3], volume.
void fem_oracle_tet(const double* Xr, const double* x, double* c, double* G, double* R, double* vol) {
  V3<double> X4[4], x4[4];
  for (int a = 0; a < 4; ++a) {
    X4[a] = V3<double>{Xr[3 * a], Xr[3 * a + 1], Xr[3 * a + 2]};
    x4[a] = V3<double>{x[3 * a], x[3 * a + 1], x[3 * a + 2]};
  }
  const TetRest<double> tr = tet_rest(X4);
  V3<double> g[6][4];
  M3<double> r;
  tet_strain(x4, tr, c, g, r);
  for (int k = 0; k < 6; ++k)
    for (int a = 0; a < 4; ++a) {
      G[(k * 4 + a) * 3] = g[k][a].x;
      G[(k * 4 + a) * 3 + 1] = g[k][a].y;
      G[(k * 4 + a) * 3 + 2] = g[k][a].z;
    }
  std::memcpy(R, r.m, sizeof(r.m));
  *vol = tr.vol;
}

// Advance n_links links (one shared mesh) by n_frames frames from frame index `frame`.
// X, V: [n_links][P][3] in and out; resid: max residual of the last frame's substeps;
// mv: matrix-vector products of the last frame.  fp32 != 0 runs the same steps in float
// arithmetic (used only to size parity tolerances).
void fem_oracle_step(int n_links, int P, int NT, int ND, const double* Xrest, const int* tets,
                     const int* rows, const int* kinds, const int* fixed, const double* prm,
                     const double* cfg, long long frame, int n_frames, double* X, double* V,
                     double* resid, int* mv, int n_threads, int fp32) {
  const Mesh M{P, NT, ND, Xrest, tets, rows, kinds, fixed};
  if (fp32)
    fem_step_t<float>(n_links, M, prm, cfg, frame, n_frames, X, V, resid, mv, n_threads);
  else
    fem_step_t<double>(n_links, M, prm, cfg, frame, n_frames, X, V, resid, mv, n_threads);
}

}  // extern "C"
