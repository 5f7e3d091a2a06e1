/*
 * femlink.h -- C-ABI of the tetrahedral soft link (arXiv 1904.02833, Sec. III-A, III-B,
 * IV-A and IV-D), part of libsnakesim.so.
 *
 * A batch of soft links that share one tetrahedral mesh (the paper meshes its link with
 * TetGen into 13 cross-sections) is advanced frame by frame.  Each substep of a frame
 *   - samples the link's chamber pressure from the open-loop command of Eq. 9 at t + h
 *     (p = A clamp(sin(2 pi f t + phase) + offset, -1, 1), Pa; p > 0 drives the right
 *     chamber, p < 0 the left one),
 *   - predicts positions under gravity (first-order implicit time stepping, Sec. IV-D),
 *   - solves the compliant constraints c(q) + E lambda = 0 (Sec. IV) of
 *       tetrahedral finite elements: six corotational strains per element in Voigt order
 *         [xx yy zz yz xz xy] (tensor shears) of F = R S, c = S - I, with the element
 *         compliance E = C / (V Y), C = [1 -nu -nu; -nu 1 -nu; -nu -nu 1] (+) (1 + nu) I3
 *         (Sec. III-B, Eq. 5),
 *       actuation distance rows of the driven chamber, rest length r eps(p),
 *         eps(p) = 1 + |p| / Y (Sec. III-A, Eq. 1-2),
 *       distance rows of constant rest length for the inextensible centre layer and the
 *         fibre-held perimeter (Sec. V),
 *     by Newton steps, each a preconditioned conjugate residual (PCR) solve of the Schur
 *     system of Eq. 8, (J M^-1 J^T + E / h^2) dlambda = -(c + E lambda / h^2), with its
 *     diagonal as preconditioner (Sec. IV-D), multipliers from zero every substep; the
 *     gradient of a strain row holds R fixed (corotational linearisation);
 *   - sets velocities from the displacement, damped by exp(-d h).
 * Particle masses are lumped (Sec. IV-A): a quarter of every adjacent element's mass.
 * Particles flagged fixed are held by a rigid cap (the attachment of Eq. 6 to a body
 * that does not move).
 *
 * One CUDA thread block advances one link for a whole frame with every vector of the
 * solve in shared memory and registers.  Conventions as in snakesim.h: every call
 * returns a SimStatus, the text of the last error is in sim_last_error(), work is
 * enqueued on the handle's stream, the library owns its device buffers, is_device
 * selects device (1) or host (0) caller buffers, one host thread per handle.
 */
#ifndef FEMLINK_H_
#define FEMLINK_H_

#include <stdint.h>

#include "snakesim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct FemHandle FemHandle; /* opaque, owned by the library */

/* Kinds of distance rows. */
enum { FEM_ROW_INEXT = 0, FEM_ROW_PERIM = 1, FEM_ROW_ACT_LEFT = 2, FEM_ROW_ACT_RIGHT = 3 };

/* Limits of one link's mesh (one thread block holds a link). */
enum { FEM_MAX_PARTICLES = 1024, FEM_MAX_TETS = 1024, FEM_MAX_ROWS = 1024 };

typedef struct {
  double dt;          /* frame length, s (> 0) */
  int32_t n_sub;      /* substeps per frame (>= 1) */
  int32_t iters;      /* cap on matrix-vector products per substep (>= 0) */
  float tol;          /* normalised residual that ends the Newton loop (>= 0; 0: run to the cap) */
  int32_t pcr_iters;  /* PCR iterations per Newton step (>= 1) */
  float gravity[3];   /* m/s^2 */
} FemConfig;

typedef struct {
  float youngs;       /* Y, Pa (> 0) */
  float poisson;      /* nu, [0, 0.5) */
  float density;      /* kg/m^3 (> 0) */
  float damping;      /* d, 1/s (>= 0) */
  float alpha_inext;  /* compliance of the centre-layer rows, m/N (>= 0) */
  float alpha_perim;  /* compliance of the perimeter rows, m/N (>= 0) */
  float alpha_act;    /* compliance of the actuation rows, m/N (>= 0) */
  float press_amp;    /* A, Pa (>= 0) */
  float press_freq;   /* f, Hz */
  float press_phase;  /* rad */
  float press_offset; /* offset inside the clamp */
} FemLinkParams;

typedef struct {
  int32_t n_particles;  /* P, 4 .. FEM_MAX_PARTICLES */
  int32_t n_tets;       /* 1 .. FEM_MAX_TETS */
  int32_t n_rows;       /* 0 .. FEM_MAX_ROWS */
  const double* rest;   /* [P][3] rest positions, m (host) */
  const int32_t* tets;  /* [n_tets][4] particle ids, positive volume (host) */
  const int32_t* rows;  /* [n_rows][2] particle ids, distinct (host) */
  const int32_t* kinds; /* [n_rows] FEM_ROW_* (host) */
  const int32_t* fixed; /* [P] 1 = held (host) */
} FemMesh;

/* Creates a batch of n_links links on `mesh` (copied), all at rest at the mesh's rest
 * positions, frame index 0.  SIM_EINVAL (nothing allocated) on a bad config, mesh
 * (index out of range, size limit, non-positive element volume, a particle in no
 * element) or parameter. */
SimStatus fem_create(const FemConfig* cfg, const FemMesh* mesh, int n_links, const FemLinkParams* params,
                     void* stream, FemHandle** out);

/* Replaces the solver configuration for the following frames. */
SimStatus fem_set_config(FemHandle* h, const FemConfig* cfg);

/* Enqueues n_frames frames (one kernel launch each); the frame index advances by n_frames. */
SimStatus fem_step(FemHandle* h, int n_frames);

/* Copies out positions and velocities [n_links][P][3] (float), the largest residual over
 * the last frame's substeps [n_links] and the matrix-vector products of the last frame
 * [n_links]; any pointer may be null.  Host copies synchronise with the stream. */
SimStatus fem_get_state(FemHandle* h, float* x, float* v, float* resid, int32_t* mv, int is_device);

/* Overwrites positions and / or velocities [n_links][P][3] (either may be null). */
SimStatus fem_set_state(FemHandle* h, const float* x, const float* v, int is_device);

/* Sets the frame index (time = frame * dt). */
SimStatus fem_set_frame(FemHandle* h, int64_t frame);

/* Kernel launches enqueued by this handle so far. */
SimStatus fem_launch_count(FemHandle* h, int64_t* n);

/* Frees the handle (synchronises with its stream). */
SimStatus fem_destroy(FemHandle* h);

#ifdef __cplusplus
}
#endif

#endif /* FEMLINK_H_ */
