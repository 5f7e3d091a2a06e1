// Tetrahedral soft link (Sec. III-A, III-B, IV-A, IV-D): one thread block advances one
// link for a whole frame; every vector of the Newton + PCR solve stays on chip.
//
// Layout of a block: thread `tid` owns the elements tid + s * blockDim (s < kTPT) and
// keeps their polar rotations and PCR vectors (z, p, q, A z and the Newton increment,
// six rows each) in registers.  Shared memory holds the mesh (shape-function gradients,
// volumes, vertex ids, distance rows, the particle -> contribution-slot lists), the
// particles (positions, substep-start positions, velocities, inverse masses, M^-1 J^T v),
// the elements' multipliers and inverse diagonals, and all vectors of the distance rows.
//
// A product y = (J M^-1 J^T + E / h^2) v runs in three phases separated by barriers:
//  A. every row writes its gradient times v into its contribution slots (element e,
//     vertex a: R Sigma(v_e) g_a; distance row d: -n v_d, +n v_d);
//  B. every particle sums its slots in a fixed order and scales by its inverse mass;
//  C. every row reads the sums at its particles: element rows Voigt(sym(R^T H)) with
//     H = sum_a u_a g_a^T, distance rows n . (u_j - u_i); plus the compliance term.
// Dot products are block reductions summed in a fixed order, so a run is reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "femlink.h"
#include "internal.h"

namespace {

constexpr int kTPT = 2;           // elements per thread
constexpr int kMaxThreads = 512;  // FEM_MAX_TETS / kTPT
constexpr int kPolarIters = 12;

SimStatus ffail(SimStatus s, const std::string& msg) {
  snakesim::set_last_error(msg.c_str());
  return s;
}

#define FCU(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return ffail(e_ == cudaErrorMemoryAllocation ? SIM_ENOMEM : SIM_ECUDA,           \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

// Offsets (in elements of each type) of the shared-memory areas of one block.
struct FemLayout {
  // floats (per-element and per-row records padded to an odd number of words: 13 per
  // element's contribution slots, 7 per element's multipliers / inverse diagonals, 7 per
  // distance row's slots, so that consecutive threads hit distinct banks)
  int g, scl, lam, idg, cont, xs, xx, vv, uu, wn, dn, drest, dat, did, dlam, ddl, dz, dp, dq, daz, red, n_float;
  // unsigned shorts (after the floats)
  int tet, row, coff, csr, n_short;
  // bytes (after the shorts)
  int kind, act, n_byte;
  size_t bytes;
  __host__ __device__ FemLayout(int P, int NT, int ND, int nnz) {
    int o = 0;
    g = o; o += NT * 9;
    scl = o; o += NT;  // compliance scale 1 / (V Y h^2) per element
    lam = o; o += NT * 7;
    idg = o; o += NT * 7;
    cont = o; o += 13 * NT + 7 * ND;  // element e vertex a comp k at 13 e + 3 a + k; row d end k at 13 NT + 7 d + 3 k
    xs = o; o += P * 3;
    xx = o; o += P * 3;
    vv = o; o += P * 3;
    uu = o; o += P * 3;
    wn = o; o += P;
    dn = o; o += ND * 3;
    drest = o; o += ND;
    dat = o; o += ND;
    did = o; o += ND;
    dlam = o; o += ND;
    ddl = o; o += ND;
    dz = o; o += ND;
    dp = o; o += ND;
    dq = o; o += ND;
    daz = o; o += ND;
    red = o; o += 64;
    o = (o + 3) & ~3;  // the vertex ids that follow are read as 8-byte words
    n_float = o;
    int s = 0;
    tet = s; s += NT * 4;
    row = s; s += ND * 2;
    coff = s; s += P + 1;
    csr = s; s += nnz;
    n_short = s;
    int b = 0;
    kind = b; b += ND;
    act = b; b += ND;
    n_byte = b;
    bytes = (size_t)n_float * 4 + (size_t)n_short * 2 + (size_t)n_byte;
    bytes = (bytes + 15) & ~(size_t)15;
  }
};

struct FemArgs {
  const float* g;             // [NT][9] shape-function gradients of vertices 1..3 (g0 = -sum)
  const float* vol;           // [NT] rest volumes
  const unsigned short* tet;  // [NT][4]
  const unsigned short* row;  // [ND][2]
  const unsigned char* kind;  // [ND]
  const float* rest;          // [ND] rest lengths
  const float* vnode;         // [P] lumped volume of each particle (sum of V / 4)
  const unsigned char* fixed; // [P]
  const unsigned short* coff; // [P + 1] first slot of each particle's list
  const unsigned short* csr;  // [nnz] contribution offsets (component 0) in slot order
  const FemLinkParams* prm;   // [links]
  float* x;                   // [links][P][3]
  float* v;                   // [links][P][3]
  float* resid;               // [links]
  int* mv;                    // [links]
  int P, NT, ND, nnz;
  long long frame;
  double dt;
  int n_sub, K, pcr_iters;
  float tol;
  float gx, gy, gz;
};

__device__ __forceinline__ float fin_or_inf(float a) { return (a <= 3.0e38f) ? a : INFINITY; }

// Sum / maximum over the block; every thread gets the same value (the per-warp partials
// combined by the same butterfly in every warp).  Consecutive reductions alternate between two halves of `red`, so one
// barrier per reduction suffices: a half is rewritten two reductions later, after every
// thread has passed the barrier of the reduction in between.
__device__ __forceinline__ float block_sum(float a, float* red, int& k) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float* r = red + 32 * (k & 1);
  ++k;
  if ((threadIdx.x & 31) == 0) r[w] = a;
  __syncthreads();
  float s = (threadIdx.x & 31) < nw ? r[threadIdx.x & 31] : 0.f;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

__device__ __forceinline__ float block_max(float a, float* red, int& k) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float* r = red + 32 * (k & 1);
  ++k;
  if ((threadIdx.x & 31) == 0) r[w] = a;
  __syncthreads();
  float s = (threadIdx.x & 31) < nw ? r[threadIdx.x & 31] : 0.f;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s = fmaxf(s, __shfl_xor_sync(0xffffffffu, s, o));
  return s;
}

// Rotation of the polar decomposition F = R S by the scaled Newton iteration
// X <- (gamma X + X^-T / gamma) / 2, gamma = |det X|^(-1/3) (Higham).  Returns false when
// det F <= 0 (an inverted element has no rotation).
__device__ __forceinline__ bool polar_rotation(const float (&F)[9], float (&R)[9]) {
  float X[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) X[i] = F[i];
  bool ok = true;
  for (int it = 0; it < kPolarIters; ++it) {
    const float c00 = X[4] * X[8] - X[5] * X[7], c01 = X[5] * X[6] - X[3] * X[8], c02 = X[3] * X[7] - X[4] * X[6];
    const float c10 = X[2] * X[7] - X[1] * X[8], c11 = X[0] * X[8] - X[2] * X[6], c12 = X[1] * X[6] - X[0] * X[7];
    const float c20 = X[1] * X[5] - X[2] * X[4], c21 = X[2] * X[3] - X[0] * X[5], c22 = X[0] * X[4] - X[1] * X[3];
    const float det = X[0] * c00 + X[1] * c01 + X[2] * c02;
    if (it == 0 && !(det > 0.f)) { ok = false; break; }
    const float gm = rcbrtf(fabsf(det));
    const float a = 0.5f * gm, b = 0.5f / (gm * det);
    const float C[9] = {c00, c01, c02, c10, c11, c12, c20, c21, c22};
    float diff = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float xn = a * X[i] + b * C[i];
      diff += fabsf(xn - X[i]);
      X[i] = xn;
    }
    if (diff < 1e-6f) break;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = X[i];
  return ok;
}

// Contribution slots of one element for a Voigt vector v: c_a = R Sigma(v) g_a (a = 1..3),
// c_0 = -(c_1 + c_2 + c_3), vertex a's three components at cont[3 a].
__device__ __forceinline__ void tet_scatter(const float (&R)[9], const float* g, const float (&v)[6], float* cont) {
  const float s00 = v[0], s11 = v[1], s22 = v[2], s12 = 0.5f * v[3], s02 = 0.5f * v[4], s01 = 0.5f * v[5];
  float t0x = 0.f, t0y = 0.f, t0z = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float gx = g[3 * a], gy = g[3 * a + 1], gz = g[3 * a + 2];
    const float sx = s00 * gx + s01 * gy + s02 * gz;
    const float sy = s01 * gx + s11 * gy + s12 * gz;
    const float sz = s02 * gx + s12 * gy + s22 * gz;
    const float cx = R[0] * sx + R[1] * sy + R[2] * sz;
    const float cy = R[3] * sx + R[4] * sy + R[5] * sz;
    const float cz = R[6] * sx + R[7] * sy + R[8] * sz;
    cont[3 * (a + 1)] = cx;
    cont[3 * (a + 1) + 1] = cy;
    cont[3 * (a + 1) + 2] = cz;
    t0x += cx; t0y += cy; t0z += cz;
  }
  cont[0] = -t0x;
  cont[1] = -t0y;
  cont[2] = -t0z;
}

// Adds the contribution slots csr[lo..hi) in order; the offsets of four slots are read
// before their values, so the dependent shared-memory loads overlap.
__device__ __forceinline__ void slot_sum(const float* cont, const unsigned short* csr, int lo, int hi, float& sx,
                                         float& sy, float& sz) {
  int e = lo;
  for (; e + 4 <= hi; e += 4) {
    const int o0 = csr[e], o1 = csr[e + 1], o2 = csr[e + 2], o3 = csr[e + 3];
    const float a0 = cont[o0], b0 = cont[o0 + 1], c0 = cont[o0 + 2];
    const float a1 = cont[o1], b1 = cont[o1 + 1], c1 = cont[o1 + 2];
    const float a2 = cont[o2], b2 = cont[o2 + 1], c2 = cont[o2 + 2];
    const float a3 = cont[o3], b3 = cont[o3 + 1], c3 = cont[o3 + 2];
    sx += a0; sy += b0; sz += c0;
    sx += a1; sy += b1; sz += c1;
    sx += a2; sy += b2; sz += c2;
    sx += a3; sy += b3; sz += c3;
  }
  for (; e < hi; ++e) {
    const float* c = cont + csr[e];
    sx += c[0]; sy += c[1]; sz += c[2];
  }
}

// Element rows of J u: Voigt(sym(R^T H)), H = sum_{a=1..3} (u_a - u_0) g_a^T.
__device__ __forceinline__ void tet_rows(const float (&R)[9], const float* g, const float* uu, ushort4 id4,
                                         float (&y)[6]) {
  const int ids[4] = {id4.x, id4.y, id4.z, id4.w};
  const float u0x = uu[3 * ids[0]], u0y = uu[3 * ids[0] + 1], u0z = uu[3 * ids[0] + 2];
  float H[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int p = ids[a + 1];
    const float dx = uu[3 * p] - u0x, dy = uu[3 * p + 1] - u0y, dz = uu[3 * p + 2] - u0z;
    const float gx = g[3 * a], gy = g[3 * a + 1], gz = g[3 * a + 2];
    H[0] += dx * gx; H[1] += dx * gy; H[2] += dx * gz;
    H[3] += dy * gx; H[4] += dy * gy; H[5] += dy * gz;
    H[6] += dz * gx; H[7] += dz * gy; H[8] += dz * gz;
  }
  float M[9];  // R^T H
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[3 * i + j] = R[i] * H[j] + R[3 + i] * H[3 + j] + R[6 + i] * H[6 + j];
  y[0] = M[0];
  y[1] = M[4];
  y[2] = M[8];
  y[3] = 0.5f * (M[5] + M[7]);
  y[4] = 0.5f * (M[2] + M[6]);
  y[5] = 0.5f * (M[1] + M[3]);
}

// (C v)_k of the element compliance pattern.
__device__ __forceinline__ void compliance(float nu, const float (&v)[6], float (&o)[6]) {
  o[0] = v[0] - nu * (v[1] + v[2]);
  o[1] = v[1] - nu * (v[0] + v[2]);
  o[2] = v[2] - nu * (v[0] + v[1]);
  o[3] = (1.f + nu) * v[3];
  o[4] = (1.f + nu) * v[4];
  o[5] = (1.f + nu) * v[5];
}

__global__ void __launch_bounds__(kMaxThreads, 1) fem_frame_kernel(FemArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const FemLayout L(A.P, A.NT, A.ND, A.nnz);
  float* fs = reinterpret_cast<float*>(smem_raw);
  unsigned short* us = reinterpret_cast<unsigned short*>(fs + L.n_float);
  unsigned char* ub = reinterpret_cast<unsigned char*>(us + L.n_short);
  float *gS = fs + L.g, *scS = fs + L.scl, *lamT = fs + L.lam, *idT = fs + L.idg, *cont = fs + L.cont;
  float *xs = fs + L.xs, *xx = fs + L.xx, *vv = fs + L.vv, *uu = fs + L.uu, *wn = fs + L.wn;
  float *dn = fs + L.dn, *drest = fs + L.drest, *dat = fs + L.dat, *did = fs + L.did, *dlam = fs + L.dlam;
  float *ddl = fs + L.ddl, *dz = fs + L.dz, *dp = fs + L.dp, *dq = fs + L.dq, *daz = fs + L.daz, *red = fs + L.red;
  unsigned short *tetS = us + L.tet, *rowS = us + L.row, *coff = us + L.coff, *csr = us + L.csr;
  unsigned char *kindS = ub + L.kind, *actS = ub + L.act;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int link = blockIdx.x;
  const int P = A.P, NT = A.NT, ND = A.ND;
  const FemLinkParams pr = A.prm[link];
  const float Y = pr.youngs, nu = pr.poisson;
  const float h = (float)(A.dt / A.n_sub);
  const float h2 = h * h;

  // ---- mesh and state of this link into shared memory; per element the compliance
  // scale 1 / (V Y h^2) of its rows (E / h^2 = scale x C)
  for (int i = tid; i < NT * 9; i += nthr) gS[i] = A.g[i];
  for (int i = tid; i < NT; i += nthr) scS[i] = 1.f / (A.vol[i] * Y * h2);
  for (int i = tid; i < NT * 4; i += nthr) tetS[i] = A.tet[i];
  for (int i = tid; i < ND * 2; i += nthr) rowS[i] = A.row[i];
  for (int i = tid; i < ND; i += nthr) kindS[i] = A.kind[i];
  for (int i = tid; i <= P; i += nthr) coff[i] = A.coff[i];
  for (int i = tid; i < A.nnz; i += nthr) csr[i] = A.csr[i];
  const float* xg = A.x + (size_t)link * P * 3;
  const float* vg = A.v + (size_t)link * P * 3;
  for (int i = tid; i < P * 3; i += nthr) { xx[i] = xg[i]; vv[i] = vg[i]; }
  for (int i = tid; i < P; i += nthr) wn[i] = A.fixed[i] ? 0.f : 1.f / (pr.density * A.vnode[i]);
  __syncthreads();

  const float damp = expf(-pr.damping * h);
  float r_frame = 0.f;
  int mv_frame = 0;
  int nred = 0;  // reductions so far (selects the half of `red`)

  float R[kTPT][9], z[kTPT][6], p[kTPT][6], q[kTPT][6], dl[kTPT][6], az[kTPT][6];

  // y = A v for v = z (element rows from registers, distance rows from dz): phases A-C.
  // Writes A z into az (elements) and daz (distance rows).
  auto product = [&](bool elements_from_dl) {
    // A: contribution slots
#pragma unroll
    for (int s = 0; s < kTPT; ++s) {
      const int t = tid + s * nthr;
      if (t < NT) {
        float vin[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) vin[k] = elements_from_dl ? dl[s][k] : z[s][k];
        tet_scatter(R[s], gS + 9 * t, vin, cont + 13 * t);
      }
    }
    for (int d = tid; d < ND; d += nthr) {
      const float vd = elements_from_dl ? ddl[d] : dz[d];
      float* c = cont + 13 * NT + 7 * d;
      const float nx = dn[3 * d] * vd, ny = dn[3 * d + 1] * vd, nz = dn[3 * d + 2] * vd;
      c[0] = -nx; c[1] = -ny; c[2] = -nz;
      c[3] = nx; c[4] = ny; c[5] = nz;
    }
    __syncthreads();
    // B: particle sums, times the inverse mass.  With at least two threads per particle,
    // threads 2i and 2i+1 each add one half of particle i's list (first half + second
    // half, a fixed order); otherwise one thread adds the whole list.
    if (2 * P <= nthr) {
      const int i = tid >> 1;
      float sx = 0.f, sy = 0.f, sz = 0.f;
      if (i < P) {
        const int b = coff[i], e1 = coff[i + 1], mid = b + (e1 - b + 1) / 2;
        slot_sum(cont, csr, (tid & 1) ? mid : b, (tid & 1) ? e1 : mid, sx, sy, sz);
      }
      sx += __shfl_xor_sync(0xffffffffu, sx, 1);
      sy += __shfl_xor_sync(0xffffffffu, sy, 1);
      sz += __shfl_xor_sync(0xffffffffu, sz, 1);
      if (i < P && (tid & 1) == 0) {
        const float w = wn[i];
        uu[3 * i] = w * sx; uu[3 * i + 1] = w * sy; uu[3 * i + 2] = w * sz;
      }
    } else {
      for (int i = tid; i < P; i += nthr) {
        float sx = 0.f, sy = 0.f, sz = 0.f;
        slot_sum(cont, csr, coff[i], coff[i + 1], sx, sy, sz);
        const float w = wn[i];
        uu[3 * i] = w * sx; uu[3 * i + 1] = w * sy; uu[3 * i + 2] = w * sz;
      }
    }
    __syncthreads();
  };
  auto rows_of_u = [&]() {
    // C: rows read the particle sums
#pragma unroll
    for (int s = 0; s < kTPT; ++s) {
      const int t = tid + s * nthr;
      if (t < NT) {
        float y[6], cz[6];
        tet_rows(R[s], gS + 9 * t, uu, reinterpret_cast<const ushort4*>(tetS)[t], y);
        compliance(nu, z[s], cz);
        const float sc = scS[t];
#pragma unroll
        for (int k = 0; k < 6; ++k) az[s][k] = y[k] + sc * cz[k];
      }
    }
    for (int d = tid; d < ND; d += nthr) {
      float y = 0.f;
      if (actS[d]) {
        const int i = rowS[2 * d], j = rowS[2 * d + 1];
        y = dn[3 * d] * (uu[3 * j] - uu[3 * i]) + dn[3 * d + 1] * (uu[3 * j + 1] - uu[3 * i + 1]) +
            dn[3 * d + 2] * (uu[3 * j + 2] - uu[3 * i + 2]) + dat[d] * dz[d];
      }
      daz[d] = y;
    }
  };

  for (int sub = 0; sub < A.n_sub; ++sub) {
    // ---- chamber pressure of Eq. 9 at the end of the substep
    const double tp = (double)(A.frame * A.n_sub + sub + 1) * (A.dt / A.n_sub);
    const double ph = fmod(2.0 * M_PI * (double)pr.press_freq * tp + (double)pr.press_phase, 2.0 * M_PI);
    const float u = fminf(1.f, fmaxf(-1.f, sinf((float)ph) + pr.press_offset));
    const float pres = pr.press_amp * u;
    const int active = pres > 0.f ? FEM_ROW_ACT_RIGHT : (pres < 0.f ? FEM_ROW_ACT_LEFT : -1);
    const float eps = 1.f + fabsf(pres) / Y;
    // ---- prediction
    for (int i = tid; i < P; i += nthr) {
      const float w = wn[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float gk = k == 0 ? A.gx : (k == 1 ? A.gy : A.gz);
        xs[3 * i + k] = xx[3 * i + k];
        if (w > 0.f) {
          vv[3 * i + k] += h * gk;
          xx[3 * i + k] += h * vv[3 * i + k];
        }
      }
    }
    for (int d = tid; d < ND; d += nthr) {
      const int kd = kindS[d];
      const bool actk = kd == FEM_ROW_INEXT || kd == FEM_ROW_PERIM || kd == active;
      const int i = rowS[2 * d], j = rowS[2 * d + 1];
      actS[d] = (actk && wn[i] + wn[j] > 0.f) ? 1 : 0;
      const float a = kd == FEM_ROW_INEXT ? pr.alpha_inext : (kd == FEM_ROW_PERIM ? pr.alpha_perim : pr.alpha_act);
      dat[d] = a / h2;
      drest[d] = (kd == FEM_ROW_ACT_LEFT || kd == FEM_ROW_ACT_RIGHT) ? A.rest[d] * eps : A.rest[d];
      dlam[d] = 0.f;
    }
    for (int i = tid; i < NT * 7; i += nthr) lamT[i] = 0.f;
    __syncthreads();

    int mv = 0;
    float r_sub = 0.f;
    for (;;) {
      // ---- linearise at x: rotations, strains, inverse diagonals, right-hand side
      float rloc = 0.f;
#pragma unroll
      for (int s = 0; s < kTPT; ++s) {
        const int t = tid + s * nthr;
        if (t < NT) {
          const ushort4 id4 = reinterpret_cast<const ushort4*>(tetS)[t];  // one 8-byte load
          const int id[4] = {id4.x, id4.y, id4.z, id4.w};
          const float* g = gS + 9 * t;
          const float x0 = xx[3 * id[0]], y0 = xx[3 * id[0] + 1], z0 = xx[3 * id[0] + 2];
          float F[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const int pa = id[a + 1];
            const float ex = xx[3 * pa] - x0, ey = xx[3 * pa + 1] - y0, ez = xx[3 * pa + 2] - z0;
            const float gx = g[3 * a], gy = g[3 * a + 1], gz = g[3 * a + 2];
            F[0] += ex * gx; F[1] += ex * gy; F[2] += ex * gz;
            F[3] += ey * gx; F[4] += ey * gy; F[5] += ey * gz;
            F[6] += ez * gx; F[7] += ez * gy; F[8] += ez * gz;
          }
          const bool ok = polar_rotation(F, R[s]);
          float M[9];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
              M[3 * i + j] = R[s][i] * F[j] + R[s][3 + i] * F[3 + j] + R[s][6 + i] * F[6 + j];
          const float c[6] = {M[0] - 1.f, M[4] - 1.f, M[8] - 1.f, 0.5f * (M[5] + M[7]), 0.5f * (M[2] + M[6]),
                              0.5f * (M[1] + M[3])};
          float lam6[6], al[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) lam6[k] = lamT[7 * t + k];
          compliance(nu, lam6, al);
          const float sc = scS[t];
          // diagonal: sum_a w_a |Sigma_k g_a|^2 + sc C_kk
          const float w0 = wn[id[0]];
          float g0x = 0.f, g0y = 0.f, g0z = 0.f;
          float dg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float gx = g[3 * a], gy = g[3 * a + 1], gz = g[3 * a + 2];
            g0x -= gx; g0y -= gy; g0z -= gz;
            const float wa = wn[id[a + 1]];
            dg[0] += wa * gx * gx; dg[1] += wa * gy * gy; dg[2] += wa * gz * gz;
            dg[3] += wa * 0.25f * (gy * gy + gz * gz);
            dg[4] += wa * 0.25f * (gx * gx + gz * gz);
            dg[5] += wa * 0.25f * (gx * gx + gy * gy);
          }
          dg[0] += w0 * g0x * g0x; dg[1] += w0 * g0y * g0y; dg[2] += w0 * g0z * g0z;
          dg[3] += w0 * 0.25f * (g0y * g0y + g0z * g0z);
          dg[4] += w0 * 0.25f * (g0x * g0x + g0z * g0z);
          dg[5] += w0 * 0.25f * (g0x * g0x + g0y * g0y);
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            const float Ckk = k < 3 ? 1.f : 1.f + nu;
            const float inv = 1.f / (dg[k] + sc * Ckk);
            idT[7 * t + k] = inv;
            const float b = -(c[k] + sc * al[k]);
            rloc = fmaxf(rloc, fin_or_inf(fabsf(b)));
            z[s][k] = b * inv;
            p[s][k] = z[s][k];
            dl[s][k] = 0.f;
          }
          if (!ok) rloc = INFINITY;
        }
      }
      for (int d = tid; d < ND; d += nthr) {
        const int i = rowS[2 * d], j = rowS[2 * d + 1];
        float ex = xx[3 * j] - xx[3 * i], ey = xx[3 * j + 1] - xx[3 * i + 1], ez = xx[3 * j + 2] - xx[3 * i + 2];
        const float len = sqrtf(ex * ex + ey * ey + ez * ez);
        const float il = 1.f / len;
        dn[3 * d] = ex * il; dn[3 * d + 1] = ey * il; dn[3 * d + 2] = ez * il;
        float zd = 0.f, inv = 0.f;
        if (actS[d]) {
          const float b = -((len - drest[d]) + dat[d] * dlam[d]);
          rloc = fmaxf(rloc, fin_or_inf(fabsf(b) / A.rest[d]));
          inv = 1.f / (wn[i] + wn[j] + dat[d]);
          zd = b * inv;
        }
        did[d] = inv;
        dz[d] = zd;
        dp[d] = zd;
        ddl[d] = 0.f;
      }
      const float r_all = block_max(rloc, red, nred);  // (its barrier also publishes dn, dz, did)
      r_sub = r_all;
      if (r_all <= A.tol || mv >= A.K) break;
      // ---- PCR from dlambda = 0 with the diagonal preconditioner
      product(false);
      rows_of_u();
      ++mv;
      float part = 0.f;
#pragma unroll
      for (int s = 0; s < kTPT; ++s)
        if (tid + s * nthr < NT)
#pragma unroll
          for (int k = 0; k < 6; ++k) { q[s][k] = az[s][k]; part += z[s][k] * az[s][k]; }
      for (int d = tid; d < ND; d += nthr) { dq[d] = daz[d]; part += dz[d] * daz[d]; }
      float zaz = block_sum(part, red, nred);
      for (int it = 0; it < A.pcr_iters && mv < A.K; ++it) {
        float qs = 0.f;
#pragma unroll
        for (int s = 0; s < kTPT; ++s) {
          const int t = tid + s * nthr;
          if (t < NT)
#pragma unroll
            for (int k = 0; k < 6; ++k) qs += q[s][k] * q[s][k] * idT[7 * t + k];
        }
        for (int d = tid; d < ND; d += nthr) qs += dq[d] * dq[d] * did[d];
        qs = block_sum(qs, red, nred);
        if (!(qs > 0.f)) break;
        const float alpha = zaz / qs;
#pragma unroll
        for (int s = 0; s < kTPT; ++s) {
          const int t = tid + s * nthr;
          if (t < NT)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              dl[s][k] += alpha * p[s][k];
              z[s][k] -= alpha * q[s][k] * idT[7 * t + k];
            }
        }
        for (int d = tid; d < ND; d += nthr) {
          ddl[d] += alpha * dp[d];
          dz[d] -= alpha * dq[d] * did[d];
        }
        // (phase A reads only this thread's rows; the particle sums it is about to
        // overwrite were last read before the barrier of the reduction above)
        product(false);
        rows_of_u();
        ++mv;
        part = 0.f;
#pragma unroll
        for (int s = 0; s < kTPT; ++s)
          if (tid + s * nthr < NT)
#pragma unroll
            for (int k = 0; k < 6; ++k) part += z[s][k] * az[s][k];
        for (int d = tid; d < ND; d += nthr) part += dz[d] * daz[d];
        const float zaz_new = block_sum(part, red, nred);
        const float beta = zaz_new / zaz;
        zaz = zaz_new;
#pragma unroll
        for (int s = 0; s < kTPT; ++s)
          if (tid + s * nthr < NT)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              p[s][k] = z[s][k] + beta * p[s][k];
              q[s][k] = az[s][k] + beta * q[s][k];
            }
        for (int d = tid; d < ND; d += nthr) {
          dp[d] = dz[d] + beta * dp[d];
          dq[d] = daz[d] + beta * dq[d];
        }
      }
      // ---- lambda += dlambda, x += M^-1 J^T dlambda
#pragma unroll
      for (int s = 0; s < kTPT; ++s) {
        const int t = tid + s * nthr;
        if (t < NT)
#pragma unroll
          for (int k = 0; k < 6; ++k) lamT[7 * t + k] += dl[s][k];
      }
      for (int d = tid; d < ND; d += nthr) dlam[d] += ddl[d];
      product(true);  // (as above: the last reduction's barrier separates the reads of uu)
      for (int i = tid; i < P * 3; i += nthr) xx[i] += uu[i];
      __syncthreads();
    }
    // ---- velocities
    const float vs = damp / h;
    for (int i = tid; i < P * 3; i += nthr) vv[i] = vs * (xx[i] - xs[i]);
    __syncthreads();
    r_frame = fmaxf(r_frame, r_sub);
    mv_frame += mv;
  }
  float* xo = A.x + (size_t)link * P * 3;
  float* vo = A.v + (size_t)link * P * 3;
  for (int i = tid; i < P * 3; i += nthr) { xo[i] = xx[i]; vo[i] = vv[i]; }
  if (tid == 0) {
    A.resid[link] = r_frame;
    A.mv[link] = mv_frame;
  }
}

// Rest data of the elements in FP64: shape-function gradients and volumes.
__global__ void fem_rest_kernel(const double* X, const int* tets, int NT, float* g, float* vol) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < NT) {
    const int* id = tets + 4 * t;
    double D[9];  // columns: x_a - x_0, a = 1..3
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) D[3 * k + a] = X[3 * id[a + 1] + k] - X[3 * id[0] + k];
    const double c00 = D[4] * D[8] - D[5] * D[7], c01 = D[5] * D[6] - D[3] * D[8], c02 = D[3] * D[7] - D[4] * D[6];
    const double c10 = D[2] * D[7] - D[1] * D[8], c11 = D[0] * D[8] - D[2] * D[6], c12 = D[1] * D[6] - D[0] * D[7];
    const double c20 = D[1] * D[5] - D[2] * D[4], c21 = D[2] * D[3] - D[0] * D[5], c22 = D[0] * D[4] - D[1] * D[3];
    const double det = D[0] * c00 + D[1] * c01 + D[2] * c02;
    // row a of D^-1 = column a of the cofactor matrix / det
    const double B[9] = {c00 / det, c10 / det, c20 / det, c01 / det, c11 / det, c21 / det,
                         c02 / det, c12 / det, c22 / det};
    for (int i = 0; i < 9; ++i) g[9 * t + i] = (float)B[i];
    vol[t] = (float)(det / 6.0);
  }
}

// Rest lengths of the distance rows in FP64.
__global__ void fem_rest_rows_kernel(const double* X, const int* rows, int ND, float* rest) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < ND) {
    const int i = rows[2 * d], j = rows[2 * d + 1];
    const double ex = X[3 * j] - X[3 * i], ey = X[3 * j + 1] - X[3 * i + 1], ez = X[3 * j + 2] - X[3 * i + 2];
    rest[d] = (float)sqrt(ex * ex + ey * ey + ez * ez);
  }
}

// Lumped volume of each particle: the sum of V / 4 over its element slots, in slot order.
__global__ void fem_node_volume_kernel(const double* X, const int* tets, const unsigned short* coff,
                                       const unsigned short* csr, int P, int NT, float* vnode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  double s = 0.0;
  for (int e = coff[i]; e < coff[i + 1]; ++e) {
    const int off = csr[e];
    if (off >= 13 * NT) continue;  // a distance row's end
    const int* id = tets + 4 * (off / 13);
    double D[9];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) D[3 * k + a] = X[3 * id[a + 1] + k] - X[3 * id[0] + k];
    const double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                       D[2] * (D[3] * D[7] - D[4] * D[6]);
    s += det / 24.0;
  }
  vnode[i] = (float)s;
}

}  // namespace

struct FemHandle {
  cudaStream_t st = nullptr;
  int n_links = 0, P = 0, NT = 0, ND = 0, nnz = 0, nthr = 0;
  size_t smem = 0;
  FemConfig cfg{};
  long long frame = 0, launches = 0;
  float *g = nullptr, *vol = nullptr, *rest = nullptr, *vnode = nullptr, *x = nullptr, *v = nullptr,
        *resid = nullptr;
  int* mv = nullptr;
  unsigned short *tet = nullptr, *row = nullptr, *coff = nullptr, *csr = nullptr;
  unsigned char *kind = nullptr, *fixed = nullptr;
  FemLinkParams* prm = nullptr;
  double* tmp_x = nullptr;  // mesh copies used only while fem_create computes the rest data
  int *tmp_t = nullptr, *tmp_r = nullptr;
};

namespace {

SimStatus validate_cfg(const FemConfig* c) {
  if (!c) return ffail(SIM_EINVAL, "null config");
  if (!(c->dt > 0.0) || c->n_sub < 1 || c->iters < 0 || !(c->tol >= 0.f) || c->pcr_iters < 1 ||
      !std::isfinite(c->gravity[0]) || !std::isfinite(c->gravity[1]) || !std::isfinite(c->gravity[2]))
    return ffail(SIM_EINVAL, "invalid config (dt > 0, n_sub >= 1, iters >= 0, tol >= 0, pcr_iters >= 1, "
                             "finite gravity)");
  return SIM_OK;
}

void free_all(FemHandle* h) {
  void* ptrs[] = {h->g,   h->vol,  h->rest, h->vnode, h->x,    h->v,     h->resid, h->mv,   h->tet,
                  h->row, h->coff, h->csr,  h->kind,  h->fixed, h->prm, h->tmp_x, h->tmp_t, h->tmp_r};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

}  // namespace

extern "C" {

SimStatus fem_create(const FemConfig* cfg, const FemMesh* mesh, int n_links, const FemLinkParams* params,
                     void* stream, FemHandle** out) {
  if (!out) return ffail(SIM_EINVAL, "null output handle");
  *out = nullptr;
  SimStatus s = validate_cfg(cfg);
  if (s != SIM_OK) return s;
  if (!mesh || !mesh->rest || !mesh->tets || !mesh->fixed || (mesh->n_rows > 0 && (!mesh->rows || !mesh->kinds)))
    return ffail(SIM_EINVAL, "null mesh array");
  const int P = mesh->n_particles, NT = mesh->n_tets, ND = mesh->n_rows;
  if (P < 4 || P > FEM_MAX_PARTICLES || NT < 1 || NT > FEM_MAX_TETS || ND < 0 || ND > FEM_MAX_ROWS)
    return ffail(SIM_EINVAL, "mesh size outside the limits (4..1024 particles, 1..1024 elements, "
                             "0..1024 distance rows)");
  if (n_links < 1 || !params) return ffail(SIM_EINVAL, "n_links < 1 or null params");
  for (int i = 0; i < 3 * P; ++i)
    if (!std::isfinite(mesh->rest[i])) return ffail(SIM_EINVAL, "non-finite rest position");
  std::vector<int> deg(P, 0);
  for (int t = 0; t < NT; ++t) {
    const int* id = mesh->tets + 4 * t;
    for (int a = 0; a < 4; ++a) {
      if (id[a] < 0 || id[a] >= P) return ffail(SIM_EINVAL, "element " + std::to_string(t) + ": vertex out of range");
      for (int b = 0; b < a; ++b)
        if (id[a] == id[b]) return ffail(SIM_EINVAL, "element " + std::to_string(t) + ": repeated vertex");
      ++deg[id[a]];
    }
    double D[9];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) D[3 * k + a] = mesh->rest[3 * id[a + 1] + k] - mesh->rest[3 * id[0] + k];
    const double det = D[0] * (D[4] * D[8] - D[5] * D[7]) - D[1] * (D[3] * D[8] - D[5] * D[6]) +
                       D[2] * (D[3] * D[7] - D[4] * D[6]);
    if (!(det > 0.0)) return ffail(SIM_EINVAL, "element " + std::to_string(t) + ": non-positive rest volume");
  }
  for (int i = 0; i < P; ++i)
    if (deg[i] == 0) return ffail(SIM_EINVAL, "particle " + std::to_string(i) + " belongs to no element");
  for (int d = 0; d < ND; ++d) {
    const int i = mesh->rows[2 * d], j = mesh->rows[2 * d + 1], k = mesh->kinds[d];
    if (i < 0 || i >= P || j < 0 || j >= P || i == j || k < 0 || k > 3)
      return ffail(SIM_EINVAL, "distance row " + std::to_string(d) + ": bad particles or kind");
    double l2 = 0.0;
    for (int c = 0; c < 3; ++c) l2 += (mesh->rest[3 * j + c] - mesh->rest[3 * i + c]) * (mesh->rest[3 * j + c] - mesh->rest[3 * i + c]);
    if (!(l2 > 0.0)) return ffail(SIM_EINVAL, "distance row " + std::to_string(d) + ": zero rest length");
  }
  for (int l = 0; l < n_links; ++l) {
    const FemLinkParams& q = params[l];
    if (!(q.youngs > 0.f) || !(q.poisson >= 0.f && q.poisson < 0.5f) || !(q.density > 0.f) || !(q.damping >= 0.f) ||
        !(q.alpha_inext >= 0.f) || !(q.alpha_perim >= 0.f) || !(q.alpha_act >= 0.f) || !(q.press_amp >= 0.f) ||
        !std::isfinite(q.press_freq) || !std::isfinite(q.press_phase) || !std::isfinite(q.press_offset))
      return ffail(SIM_EINVAL, "invalid parameters of link " + std::to_string(l) +
                                   " (Y > 0, 0 <= nu < 0.5, density > 0, damping >= 0, compliances >= 0, "
                                   "amplitude >= 0)");
  }
  // contribution slots of each particle in ascending slot order (element e vertex a: slot
  // 4 e + a, offset 13 e + 3 a; distance row d end k: slot 4 NT + 2 d + k, offset
  // 13 NT + 7 d + 3 k), stored as offsets of component 0
  const int nnz = 4 * NT + 2 * ND;
  std::vector<int> cnt(P + 1, 0);
  for (int t = 0; t < NT; ++t)
    for (int a = 0; a < 4; ++a) ++cnt[mesh->tets[4 * t + a] + 1];
  for (int d = 0; d < ND; ++d) { ++cnt[mesh->rows[2 * d] + 1]; ++cnt[mesh->rows[2 * d + 1] + 1]; }
  for (int i = 0; i < P; ++i) cnt[i + 1] += cnt[i];
  std::vector<unsigned short> coff(P + 1), csr(nnz);
  for (int i = 0; i <= P; ++i) coff[i] = (unsigned short)cnt[i];
  std::vector<int> pos(cnt.begin(), cnt.end() - 1);
  for (int t = 0; t < NT; ++t)
    for (int a = 0; a < 4; ++a) csr[pos[mesh->tets[4 * t + a]]++] = (unsigned short)(13 * t + 3 * a);
  for (int d = 0; d < ND; ++d)
    for (int k = 0; k < 2; ++k) csr[pos[mesh->rows[2 * d + k]]++] = (unsigned short)(13 * NT + 7 * d + 3 * k);
  // launch shape and shared memory
  const int nthr = ((NT + kTPT - 1) / kTPT + 31) / 32 * 32;
  const FemLayout lay(P, NT, ND, nnz);
  int dev = 0, smem_max = 0;
  FCU(cudaGetDevice(&dev));
  FCU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (lay.bytes > (size_t)smem_max)
    return ffail(SIM_EINVAL, "mesh needs " + std::to_string(lay.bytes) + " bytes of shared memory per block (" +
                                 std::to_string(smem_max) + " available)");
  FCU(cudaFuncSetAttribute(fem_frame_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes));

  FemHandle* h = new FemHandle();
  h->st = (cudaStream_t)stream;
  h->n_links = n_links; h->P = P; h->NT = NT; h->ND = ND; h->nnz = nnz; h->nthr = nthr; h->smem = lay.bytes;
  h->cfg = *cfg;
  auto cleanup = [&](SimStatus st) {
    free_all(h);
    delete h;
    return st;
  };
#define FALLOC(ptr, bytes)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes) > 0 ? (bytes) : 16);                  \
    if (e_ != cudaSuccess) return cleanup(ffail(SIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e_))); \
  } while (0)
  const size_t nstate = (size_t)n_links * P * 3;
  FALLOC(h->g, sizeof(float) * NT * 9);
  FALLOC(h->vol, sizeof(float) * NT);
  FALLOC(h->rest, sizeof(float) * ND);
  FALLOC(h->vnode, sizeof(float) * P);
  FALLOC(h->x, sizeof(float) * nstate);
  FALLOC(h->v, sizeof(float) * nstate);
  FALLOC(h->resid, sizeof(float) * n_links);
  FALLOC(h->mv, sizeof(int) * n_links);
  FALLOC(h->tet, sizeof(unsigned short) * NT * 4);
  FALLOC(h->row, sizeof(unsigned short) * ND * 2);
  FALLOC(h->coff, sizeof(unsigned short) * (P + 1));
  FALLOC(h->csr, sizeof(unsigned short) * nnz);
  FALLOC(h->kind, ND);
  FALLOC(h->fixed, P);
  FALLOC(h->prm, sizeof(FemLinkParams) * n_links);
  // rest data on the device (FP64), from temporary copies of the mesh
  FALLOC(h->tmp_x, sizeof(double) * P * 3);
  FALLOC(h->tmp_t, sizeof(int) * NT * 4);
  FALLOC(h->tmp_r, sizeof(int) * ND * 2);
  double* dX = h->tmp_x;
  int *dT = h->tmp_t, *dR = h->tmp_r;
  auto free_tmp = [&]() {
    cudaFree(h->tmp_x); cudaFree(h->tmp_t); cudaFree(h->tmp_r);
    h->tmp_x = nullptr; h->tmp_t = nullptr; h->tmp_r = nullptr;
  };
  std::vector<unsigned short> tet16(NT * 4), row16(ND * 2);
  for (int i = 0; i < NT * 4; ++i) tet16[i] = (unsigned short)mesh->tets[i];
  for (int i = 0; i < ND * 2; ++i) row16[i] = (unsigned short)mesh->rows[i];
  std::vector<unsigned char> kind8(ND), fixed8(P);
  for (int d = 0; d < ND; ++d) kind8[d] = (unsigned char)mesh->kinds[d];
  for (int i = 0; i < P; ++i) fixed8[i] = mesh->fixed[i] ? 1 : 0;
  std::vector<float> x0(nstate);
  for (int l = 0; l < n_links; ++l)
    for (int i = 0; i < 3 * P; ++i) x0[(size_t)l * P * 3 + i] = (float)mesh->rest[i];
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMemcpyAsync(dX, mesh->rest, sizeof(double) * P * 3, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(dT, mesh->tets, sizeof(int) * NT * 4, cudaMemcpyHostToDevice, h->st))) break;
    if (ND > 0 && (e = cudaMemcpyAsync(dR, mesh->rows, sizeof(int) * ND * 2, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(h->tet, tet16.data(), sizeof(unsigned short) * NT * 4, cudaMemcpyHostToDevice, h->st))) break;
    if (ND > 0 && (e = cudaMemcpyAsync(h->row, row16.data(), sizeof(unsigned short) * ND * 2, cudaMemcpyHostToDevice, h->st))) break;
    if (ND > 0 && (e = cudaMemcpyAsync(h->kind, kind8.data(), ND, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(h->fixed, fixed8.data(), P, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(h->coff, coff.data(), sizeof(unsigned short) * (P + 1), cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(h->csr, csr.data(), sizeof(unsigned short) * nnz, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(h->prm, params, sizeof(FemLinkParams) * n_links, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemcpyAsync(h->x, x0.data(), sizeof(float) * nstate, cudaMemcpyHostToDevice, h->st))) break;
    if ((e = cudaMemsetAsync(h->v, 0, sizeof(float) * nstate, h->st))) break;
    if ((e = cudaMemsetAsync(h->resid, 0, sizeof(float) * n_links, h->st))) break;
    if ((e = cudaMemsetAsync(h->mv, 0, sizeof(int) * n_links, h->st))) break;
    fem_rest_kernel<<<(NT + 127) / 128, 128, 0, h->st>>>(dX, dT, NT, h->g, h->vol);
    if ((e = cudaGetLastError())) break;
    if (ND > 0) {
      fem_rest_rows_kernel<<<(ND + 127) / 128, 128, 0, h->st>>>(dX, dR, ND, h->rest);
      if ((e = cudaGetLastError())) break;
    }
    fem_node_volume_kernel<<<(P + 127) / 128, 128, 0, h->st>>>(dX, dT, h->coff, h->csr, P, NT, h->vnode);
    if ((e = cudaGetLastError())) break;
    e = cudaStreamSynchronize(h->st);  // host staging vectors go out of scope
  } while (0);
  free_tmp();
  if (e != cudaSuccess) return cleanup(ffail(SIM_ECUDA, std::string("fem_create: ") + cudaGetErrorString(e)));
#undef FALLOC
  *out = h;
  return SIM_OK;
}

SimStatus fem_set_config(FemHandle* h, const FemConfig* cfg) {
  if (!h) return ffail(SIM_EINVAL, "null handle");
  SimStatus s = validate_cfg(cfg);
  if (s != SIM_OK) return s;
  h->cfg = *cfg;
  return SIM_OK;
}

SimStatus fem_step(FemHandle* h, int n_frames) {
  if (!h) return ffail(SIM_EINVAL, "null handle");
  if (n_frames < 0) return ffail(SIM_EINVAL, "n_frames < 0");
  FemArgs A;
  A.g = h->g; A.vol = h->vol; A.tet = h->tet; A.row = h->row; A.kind = h->kind; A.rest = h->rest;
  A.vnode = h->vnode; A.fixed = h->fixed; A.coff = h->coff; A.csr = h->csr; A.prm = h->prm;
  A.x = h->x; A.v = h->v; A.resid = h->resid; A.mv = h->mv;
  A.P = h->P; A.NT = h->NT; A.ND = h->ND; A.nnz = h->nnz;
  A.dt = h->cfg.dt; A.n_sub = h->cfg.n_sub; A.K = h->cfg.iters; A.pcr_iters = h->cfg.pcr_iters;
  A.tol = h->cfg.tol; A.gx = h->cfg.gravity[0]; A.gy = h->cfg.gravity[1]; A.gz = h->cfg.gravity[2];
  for (int f = 0; f < n_frames; ++f) {
    A.frame = h->frame;
    fem_frame_kernel<<<h->n_links, h->nthr, h->smem, h->st>>>(A);
    FCU(cudaGetLastError());
    ++h->frame;
    ++h->launches;
  }
  return SIM_OK;
}

SimStatus fem_get_state(FemHandle* h, float* x, float* v, float* resid, int32_t* mv, int is_device) {
  if (!h) return ffail(SIM_EINVAL, "null handle");
  const cudaMemcpyKind k = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const size_t ns = (size_t)h->n_links * h->P * 3;
  if (x) FCU(cudaMemcpyAsync(x, h->x, sizeof(float) * ns, k, h->st));
  if (v) FCU(cudaMemcpyAsync(v, h->v, sizeof(float) * ns, k, h->st));
  if (resid) FCU(cudaMemcpyAsync(resid, h->resid, sizeof(float) * h->n_links, k, h->st));
  if (mv) FCU(cudaMemcpyAsync(mv, h->mv, sizeof(int) * h->n_links, k, h->st));
  if (!is_device) FCU(cudaStreamSynchronize(h->st));
  return SIM_OK;
}

SimStatus fem_set_state(FemHandle* h, const float* x, const float* v, int is_device) {
  if (!h) return ffail(SIM_EINVAL, "null handle");
  const cudaMemcpyKind k = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t ns = (size_t)h->n_links * h->P * 3;
  if (x) FCU(cudaMemcpyAsync(h->x, x, sizeof(float) * ns, k, h->st));
  if (v) FCU(cudaMemcpyAsync(h->v, v, sizeof(float) * ns, k, h->st));
  if (!is_device) FCU(cudaStreamSynchronize(h->st));
  return SIM_OK;
}

SimStatus fem_set_frame(FemHandle* h, int64_t frame) {
  if (!h) return ffail(SIM_EINVAL, "null handle");
  if (frame < 0) return ffail(SIM_EINVAL, "frame < 0");
  h->frame = frame;
  return SIM_OK;
}

SimStatus fem_launch_count(FemHandle* h, int64_t* n) {
  if (!h || !n) return ffail(SIM_EINVAL, "null handle or output");
  *n = h->launches;
  return SIM_OK;
}

SimStatus fem_destroy(FemHandle* h) {
  if (!h) return ffail(SIM_EINVAL, "null handle");
  cudaStreamSynchronize(h->st);
  free_all(h);
  delete h;
  return SIM_OK;
}

}  // extern "C"
