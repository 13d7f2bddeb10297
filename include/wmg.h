/*
 * wmg.h -- C ABI of libwmg: adaptive-multigrid-preconditioned solve of the
 * Wilson-Dirac equation D(U) psi = b on one NVIDIA B300 (sm_103a).
 *
 * Method: Babich, Brannick, Brower, Clark, Cohen, Osborn, Rebbi, "The role of
 * multigrid algorithms for LQCD" (arXiv:0912.2186).
 *   Sec. 2, eq. for D_xy(U) ........ the fine operator D (wmg_apply_D)
 *   Sec. 2, P: V^ -> S, R = P^dag .. prolongation / restriction (wmg_prolong,
 *                                     wmg_restrict)
 *   Sec. 2, P = orthonormal basis of theta_xhat(x) psi^(alpha)_x ... block
 *                                     orthonormalisation inside wmg_setup
 *   Sec. 2, D^ = R D P (Galerkin) ... the coarse operator (wmg_apply_coarse)
 *   Sec. 2, adaptive construction .. wmg_setup
 *   Sec. 3 ........................... chirality split sigma_3 P = P gamma_5,
 *                                     4^4 blocks, post-smoothing cycle, GCR outer
 *                                     solver, CG on the normal equations on the
 *                                     coarsest level (wmg_solve)
 *   Sec. 4 ("multiple lattices ... interpolation and prolongation operators")
 *                                     the shape of this API.
 *
 * Conventions
 * -----------
 * * Every call returns a wmg_status; nothing throws across the ABI.  On an error
 *   the context is left usable unless the status is WMG_ECUDA, after which only
 *   wmg_destroy is valid.
 * * Lattice extents dims = {X, Y, Z, T}; direction mu = 0..3 is x, y, z, t.
 *   The lexicographic site index is x + X*(y + Y*(z + Z*t)); V = X*Y*Z*T.
 *   Boundary conditions are periodic in all four directions.
 * * Complex numbers are interleaved (re, im).
 * * Canonical layouts, used by every *_host argument and by the canonical device
 *   buffers of wmg_pack_spinor / wmg_unpack_spinor / wmg_solve_dev:
 *     gauge field  : [t][z][y][x][mu][a][b] complex double, U_mu(x)^{ab}
 *                    (the link leaving x in direction +mu; must be SU(3)).
 *     fine spinor  : [rhs][t][z][y][x][spin][colour] complex double
 *                    (component index k = 3*spin + colour).
 *     coarse field : [rhs][site][2N] complex double, coarse sites lexicographic on
 *                    the coarse lattice, coarse dof c = s*N + alpha with chirality
 *                    s = 0 (sigma_3 = +1) first.
 * * Gamma matrices (chiral basis): gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
 *   (k = 1, 2, 3 for x, y, z), gamma_4 = [[0, 1], [1, 0]] (t), so gamma_5 =
 *   diag(1, 1, -1, -1).  D psi(x) = (4 + m) psi(x)
 *     - 1/2 sum_mu [(1 - gamma_mu) U_mu(x) psi(x + mu)
 *                   + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)].
 * * Native device layouts (operator entry points):
 *     fine spinor, WMG_PREC_DOUBLE: [rhs][6][V][2] complex double
 *     fine spinor, WMG_PREC_SINGLE: [rhs][6][V][2] complex float (float4 chunks)
 *       chunk c of site v holds the components k = 2c and 2c + 1.
 *     coarse vector, both precisions: [rhs][site][2N] complex.
 *   wmg_pack_spinor / wmg_unpack_spinor convert canonical device buffers.
 * * Device pointers passed in stay owned by the caller; work is stream-ordered on
 *   the context's stream (wmg_create) and the call returns without synchronising
 *   unless its comment says otherwise.  Host buffers are read or written before the
 *   call returns.
 * * A context is not thread-safe; distinct contexts are independent.
 */
#ifndef WMG_H
#define WMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wmg_ctx wmg_ctx;

typedef enum {
  WMG_OK = 0,
  WMG_EINVAL = 1,   /* bad argument (null pointer, size, layout, precision) */
  WMG_ENOMEM = 2,   /* device or host allocation failed */
  WMG_ECUDA = 3,    /* CUDA runtime error (see wmg_last_error) */
  WMG_ENOCONV = 4,  /* solver did not reach the tolerance within max_iter */
  WMG_ERANK = 5,    /* block Gram-Schmidt found a rank-deficient block */
  WMG_ETIMEOUT = 6, /* a bounded device-side wait expired */
  WMG_ESTATE = 7    /* call order (e.g. solve before setup, no gauge loaded) */
} wmg_status;

typedef enum {
  WMG_PREC_DOUBLE = 0, /* FP64 storage and arithmetic */
  WMG_PREC_SINGLE = 1, /* FP32 storage and arithmetic */
  WMG_PREC_HALF = 2    /* FP16 storage, FP32 arithmetic: wmg_apply_coarse (FP16 operator on tensor
                          cores), wmg_restrict / wmg_prolong (FP16 null vectors), prec_nullvec,
                          prec_smoother */
} wmg_prec;

#define WMG_MAX_LEVELS 3

/* Parameters of the hierarchy and of the solve. */
typedef struct {
  int nlevels;                       /* 2 or 3 (Sec. 3 uses 3)                      */
  int block[WMG_MAX_LEVELS - 1][4];  /* block extents {bx,by,bz,bt} per coarsening
                                        (4^4 on the fine level, Sec. 3)             */
  int nvec[WMG_MAX_LEVELS - 1];      /* near-null vectors N per coarsening          */
  int setup_passes;                  /* adaptive passes (>= 1)                       */
  int setup_relax;                   /* MR steps relaxing A psi = 0 in pass 1        */
  int nu_post;                       /* post-smoothing MR steps (Sec. 3: 4)          */
  int gcr_restart;                   /* outer flexible GCR restart length            */
  int cycle_gamma;                   /* 1 = V-cycle, 2 = W-cycle at middle levels    */
  double tol;                        /* target |b - D x| / |b| (FP64 true residual)  */
  double coarse_tol;                 /* coarsest CGNR relative tolerance             */
  int coarse_maxit;                  /* coarsest CGNR iteration cap                  */
  int max_iter;                      /* outer iteration cap (cycle applications)     */
  int prec_sloppy;                   /* precision of the cycle, the hierarchy and the
                                        inner Krylov vectors (WMG_PREC_*)            */
  int coarse_tc;                     /* with prec_sloppy = SINGLE: apply the coarse
                                        stencils on FP16 tensor cores (FP32
                                        accumulation) where 2N is 16, 32, 48 or 64:
                                        1 = mma.sync, 2 = tcgen05 (TMEM accumulator),
                                        3 = autotune: after each Galerkin build, time the
                                        FP32 CUDA-core, mma.sync and tcgen05 stencils on
                                        12 rhs and keep the fastest per level            */
  double reliable_delta;             /* FP64 reliable update when the iterated
                                        residual fell by this factor                */
  uint64_t seed;                     /* seed of the setup's Gaussian starts when no
                                        starts are passed                           */
  int prec_nullvec;                  /* storage of the fine-level null vectors in the
                                        cycle's restrict / prolong with prec_sloppy =
                                        SINGLE: SINGLE, or HALF (FP16 P, FP32
                                        arithmetic; the setup keeps FP64 / FP32 P)   */
  int prec_smoother;                 /* storage of the fine-level MR smoother vectors
                                        with prec_sloppy = SINGLE: SINGLE, or HALF
                                        (FP16 with a per-site norm, FP32 arithmetic)  */
  int coarse_persistent;             /* 1: the coarsest CGNR as one cooperative
                                        persistent kernel (mma.sync stencil, 2N in
                                        {16..64}, <= 16 rhs; grid barriers bounded,
                                        WMG_ETIMEOUT when one expires); 0 (default):
                                        a device-side loop of separate launches
                                        (CUDA graph with a conditional WHILE node)   */
  int coarse_eo;                     /* 1 (default): the coarsest CG runs on the normal
                                        equations of the even-odd Schur complement
                                        S = A_ee - A_eo A_oo^-1 A_oe and recovers
                                        x_o = A_oo^-1 (b_o - A_oe x_e), same stopping
                                        test |b - A x| <= coarse_tol |b|; used where
                                        every extent of the coarsest lattice is even
                                        and 2N <= 64, else the plain CGNR; 0: plain  */
  int fine_eo;                       /* 1: red/black preconditioning of the fine solve
                                        (Sec. 3): the outer GCR runs on the even-site
                                        Schur complement S = d - H_eo H_oe / d (d = 4 +
                                        m, H the hopping term) with half-lattice Krylov
                                        vectors, the cycle of the whole lattice applied
                                        to (r_e, 0) as preconditioner, and the odd
                                        sites reconstructed, x_o = (b_o - H_oe x_e) / d;
                                        the stopping test stays |b - D x| <= tol |b|
                                        (the residual vanishes on the odd sites).  The
                                        x extent must be even.  0 (default): the whole
                                        lattice                                       */
} wmg_params;

/* Per-right-hand-side result of a solve. */
typedef struct {
  int iters;               /* outer iterations = applications of the cycle        */
  int reliable_updates;    /* FP64 true-residual recomputations                   */
  int converged;           /* 1 if true_resid <= tol                              */
  int pad_;
  double true_resid;       /* |b - D x| / |b| computed in FP64 on the device       */
  double seconds;          /* wall time of the whole (batched) solve              */
} wmg_info;

/* Fill *p with the defaults: 2 levels, 4^4 then 2^4 blocks, N = 24 then 32, 5 setup passes with
 * 100 MR relaxation steps in pass 1, nu_post = 4, FGCR(16), V-cycle, tol 1e-10, coarse_tol 0.1,
 * coarse_maxit 2000, max_iter 1000, FP32 cycle with mma.sync coarse stencils, reliable_delta 1e-4,
 * FP32 null vectors and smoother, the even-odd coarsest CG.  (On the 16^3x32 field at
 * lambda_min(D^dag D) = 1e-3 .. 1e-5 m^2, 100 relaxation steps instead of 20 keep the outer
 * iteration count within 1.4x across the three masses, 38 / 47 / 53 instead of 45 / 75 / 142.) */
void wmg_default_params(wmg_params* p);

const char* wmg_strerror(wmg_status s);
/* Text of the last error seen by this context (or ""). */
const char* wmg_last_error(const wmg_ctx* ctx);

/* Create a context for an X*Y*Z*T lattice working on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  Every extent must be >= 2.
 * The context owns all device memory it allocates. */
wmg_status wmg_create(wmg_ctx** out, const int dims[4], void* cuda_stream);
wmg_status wmg_destroy(wmg_ctx* ctx);

/* Load U (canonical layout, V*4*9 complex double).  Keeps the 12-real compressed
 * form (rows 0 and 1; row 2 = conj(row0 x row1) is rebuilt on use, Table 2's "12
 * floats") in FP64 and FP32.  Drops any hierarchy.  Host variant synchronises. */
wmg_status wmg_load_gauge(wmg_ctx* ctx, const double* U_host);
wmg_status wmg_load_gauge_dev(wmg_ctx* ctx, const double* U_dev);

/* Link storage of the FP32 fine operator (the cycle's smoother and the sloppy Krylov operator):
 * 12 reals (rows 0 and 1, row 2 = conj(row0 x row1); the default) or 8 reals (Table 2's "8
 * floats"): elements (0,1), (0,2), (1,0) and the phases of (0,0) and (2,0), the rest rebuilt from
 * unitarity and det U = 1 (moduli from the row-0 and column-0 norms, (1,1), (1,2), (2,1), (2,2) by
 * Cramer's rule from row orthogonality and the cofactor relations of U^-1 = U^dag).  The 8-real
 * links are made from the FP64 links at every gauge load; FP64 operators, the Galerkin product and
 * the no-alloc residual keep 12 reals.  A field with a link whose (0,1) and (0,2) elements (nearly)
 * vanish, |U_01|^2 + |U_02|^2 < 1e-6 (the free field, for one), is not representable that way: for
 * such a field the FP32 operator keeps the 12-real links.  reals = 18 stores all nine elements
 * in FP32 (row 2 rebuilt once, in FP64, at the gauge load): 50 % more link bytes than 12 reals
 * and no arithmetic on load.  reals: 18, 12 or 8, else WMG_EINVAL.  Synchronises when a field is
 * loaded. */
wmg_status wmg_set_gauge_compression(wmg_ctx* ctx, int reals);

/* Set the Wilson mass m (Sec. 2, the (4 + m) term).  An existing hierarchy's coarse
 * operators are shifted by (m - m_setup) on their diagonal blocks, which is exact
 * because P^dag P = 1. */
wmg_status wmg_set_mass(wmg_ctx* ctx, double m);

/* Adaptive setup (Sec. 2): near-null vectors, block orthonormalisation with the
 * chirality split of Sec. 3, Galerkin coarse operators, level by level.
 * starts_host: NULL or, for the fine level, nvec[0] fine spinors in the canonical
 * layout.  NULL draws Gaussian starts on the device from the counter-based Philox-4x32-10
 * generator keyed by p->seed (p->seed + 1 for the second level; Box-Muller in FP32), real
 * and imaginary parts in canonical order.  Synchronises. */
wmg_status wmg_setup(wmg_ctx* ctx, const wmg_params* p, const double* starts_host);

/* Setup amortisation across gauge updates (Sec. 4: the coarse operators of a slowly evolving
 * field, as in HMC, reuse the near-null subspace for several steps with an incremental update).
 * wmg_update_gauge loads a new U (canonical layout, as wmg_load_gauge) but keeps the hierarchy's
 * block-orthonormal vectors P of every level and rebuilds only the Galerkin coarse operators
 * D^ = P^dag D(U_new) P (at the setup's mass).  wmg_refresh_setup then runs `passes` improvement
 * passes of the adaptive setup on the current field, level by level, from the current subspace
 * (the starting vectors are the N fields of P, field k holding basis vector k of every block):
 * psi_k <- K(psi_k) with the two-level cycle of the current hierarchy, normalised, P and D^ rebuilt
 * after each pass.  WMG_ESTATE without a hierarchy, or when only FP16 fine null vectors are kept
 * (prec_nullvec HALF; set up again instead).  Both synchronise. */
wmg_status wmg_update_gauge(wmg_ctx* ctx, const double* U_host);
wmg_status wmg_update_gauge_dev(wmg_ctx* ctx, const double* U_dev);
wmg_status wmg_refresh_setup(wmg_ctx* ctx, int passes);

/* Replace the near-null vectors of `level` (0: fine spinors, canonical layout;
 * 1: coarse fields of the level-1 lattice) by the given host vectors, then
 * block-orthonormalise them and rebuild the coarse operators from that level down.
 * p gives the parameters (NULL: those of the last setup).  Synchronises. */
wmg_status wmg_import_nullvecs(wmg_ctx* ctx, const wmg_params* p, int level, const double* host);
/* Copy the block-orthonormalised vectors P of `level` to host (same layout).      */
wmg_status wmg_export_nullvecs(wmg_ctx* ctx, int level, double* host);
/* Copy the coarse operator of lattice level+1 (FP64) to host as
 * [site][9][2N][2N] complex double, slot k = 0 self, 1 + 2 mu + (0: +mu, 1: -mu),
 * row-major blocks: (D^ phi)(xhat) = sum_k D^[xhat][k] phi(xhat + k).  Synchronises. */
wmg_status wmg_export_coarse(wmg_ctx* ctx, int level, double* host);
/* Stencil implementation the FP32 cycle uses on coarse `level` (0 CUDA cores FP32,
 * 1 mma.sync FP16, 2 tcgen05 FP16) and, with coarse_tc = 3, the autotuner's times in ms per
 * 12-rhs launch of each (0 where not available); ms may be NULL. */
wmg_status wmg_coarse_impl(const wmg_ctx* ctx, int level, int* impl, float ms[3]);
/* Device bytes the context holds now (links in FP64 and FP32, every copy of the transfer and
 * coarse operators, solver workspaces grown so far, reduction buffers). */
wmg_status wmg_device_bytes(const wmg_ctx* ctx, size_t* bytes);
/* Number of sites and of complex dof per site of lattice `level` (0 = fine). */
wmg_status wmg_level_info(const wmg_ctx* ctx, int level, int* nsites, int* ndof);

/* Solve D x = b for nrhs right-hand sides with MG-preconditioned flexible GCR
 * (Sec. 3) to |b - D x| <= tol |b| in FP64.  b, x: canonical fine spinors.  Every
 * right-hand side is iterated independently (its result does not depend on the
 * others in the batch).  info: array of nrhs or NULL.  Returns WMG_ENOCONV if any
 * right-hand side missed the tolerance.  Both variants synchronise. */
wmg_status wmg_solve(wmg_ctx* ctx, const double* b_host, double* x_host, int nrhs, wmg_info* info);
wmg_status wmg_solve_dev(wmg_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, wmg_info* info);
/* The same outer solver without preconditioner (FP64), for comparison. */
wmg_status wmg_solve_plain_dev(wmg_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, wmg_info* info);
/* Unpreconditioned baseline (the CG of Sec. 3's comparison, on the normal equations): CG on
 * D^dag D x = D^dag b in FP64 (CGLS form; D^dag = gamma_5 D gamma_5) at the context's mass, each
 * right-hand side to |b - D x| <= tol |b| (tol of the last setup, else 1e-10) with the true
 * residual checked at the end and the iteration restarted from x while it is above tol.  Needs
 * only the gauge field (no hierarchy).  b, x: canonical device spinors.  info[k].iters = CG
 * iterations (two operator applications each), info[k].reliable_updates = true-residual
 * evaluations.  maxit caps the CG iterations; WMG_ENOCONV if a right-hand side missed tol within
 * it.  Synchronises. */
wmg_status wmg_solve_cgnr_dev(wmg_ctx* ctx, const double* b_dev, double* x_dev, int nrhs, int maxit, wmg_info* info);

/* ---- operator-level entry points (native device layouts, stream-ordered) ---- */

/* canonical [rhs][V][12] complex double  <->  native fine spinor of precision prec */
wmg_status wmg_pack_spinor(wmg_ctx* ctx, int prec, const double* canon_dev, void* native_dev, int nrhs);
wmg_status wmg_unpack_spinor(wmg_ctx* ctx, int prec, const void* native_dev, double* canon_dev, int nrhs);

/* out = D(U) in for nrhs native fine spinors (Sec. 2, eq. for D) at the context's
 * mass.  in and out must not overlap.  prec = WMG_PREC_HALF takes FP32 buffers and runs
 * the smoother's FP16 storage path: in rounded to FP16 with a per-site norm, D applied
 * in FP32 arithmetic, the result rounded to FP16 the same way and widened into out. */
wmg_status wmg_apply_D(wmg_ctx* ctx, int prec, const void* in_dev, void* out_dev, int nrhs);

/* out = S in on the even sites (odd sites of out set to 0, those of in not read): the even-site
 * Schur complement S = d - H_eo H_oe / d of the fine operator (d = 4 + m at the context's mass, H
 * the hopping term, parity (x + y + z + t) mod 2), the operator of the red/black solve (fine_eo);
 * native fine spinors of precision prec (DOUBLE or SINGLE).  The x extent must be even. */
wmg_status wmg_apply_D_eo(wmg_ctx* ctx, int prec, const void* in_dev, void* out_dev, int nrhs);

/* out = K(in): one application of the multigrid preconditioner of the fine level (Sec. 3: the
 * cycle the outer GCR applies each iteration) to nrhs native fine spinors of precision prec
 * (DOUBLE or SINGLE) at the context's mass: restrict with P^dag, the coarse solve (CG on the
 * normal equations on the coarsest level, to coarse_tol) or, with 3 levels, the next cycle
 * (cycle_gamma times at the middle level: the W-cycle for 2), prolong with P, then nu_post MR
 * steps on D out = in from the prolonged correction (post-smoothing only).  SINGLE uses the
 * hierarchy's FP32 operators (and its tensor-core coarse stencil, FP16 null vectors or FP16
 * smoother storage where configured); DOUBLE its FP64 operators.  in and out must not overlap.
 * WMG_ESTATE without a hierarchy, or for DOUBLE / SINGLE when only FP16 fine null vectors are
 * kept. */
wmg_status wmg_apply_cycle(wmg_ctx* ctx, int prec, const void* in_dev, void* out_dev, int nrhs);
/* The smoother of the cycle on its own (Sec. 3, "post smoothing iterations"): nu steps of
 * minimal-residual relaxation of D x = b on the fine level for nrhs native fine spinors of
 * precision prec, in place on x (its contents are the initial guess): r = b - D x, then nu
 * times q = D r, alpha = <q, r> / <q, q>, x += alpha r, r -= alpha q.  With prec SINGLE and a
 * hierarchy set up with prec_smoother HALF, r and q are stored in FP16 as in the cycle.  b and
 * x must not overlap. */
wmg_status wmg_smooth(wmg_ctx* ctx, int prec, const void* b_dev, void* x_dev, int nrhs, int nu);

/* coarse = P^dag fine (Sec. 2, R = P^dag): level 0 maps native fine spinors to
 * level-1 coarse vectors, level 1 maps level-1 to level-2 coarse vectors.  prec is
 * the precision of both buffers (the hierarchy must hold P in it). */
wmg_status wmg_restrict(wmg_ctx* ctx, int level, int prec, const void* fine_dev, void* coarse_dev, int nrhs);
/* fine = P coarse (Sec. 2). */
wmg_status wmg_prolong(wmg_ctx* ctx, int level, int prec, const void* coarse_dev, void* fine_dev, int nrhs);
/* out = D^ in on coarse lattice `level` >= 1 (Sec. 2 Galerkin operator), or
 * sigma_3 D^ sigma_3 = D^dag (Sec. 3) if dagger != 0.  prec = WMG_PREC_HALF applies the FP16
 * tensor-core copy of the operator to FP32 vectors (requires coarse_tc and 2N in {16..64}). */
wmg_status wmg_apply_coarse(wmg_ctx* ctx, int level, int prec, int dagger, const void* in_dev, void* out_dev,
                            int nrhs);
/* out = S in with S = D^_ee - D^_eo D^_oo^-1 D^_oe the even-odd Schur complement of the coarse
 * operator of `level` at the context's mass (the operator of the coarsest CG with coarse_eo),
 * or S^dag = sigma_3 S sigma_3 if dagger != 0.  Parity of a site: (x + y + z + t) mod 2, even
 * = 0.  Vectors [rhs][site][2N] over the whole coarse lattice: the odd-site entries of in are
 * not read, those of out are set to 0.  prec: DOUBLE or SINGLE (CUDA-core stencil, D^_oo^-1 in
 * that precision from an FP64 inversion) or HALF (FP16 tensor-core stencil copy, FP32 vectors
 * and inverse).  WMG_EINVAL if an extent of the level is odd or 2N > 64; WMG_ERANK if a site
 * block of D^_oo is singular. */
wmg_status wmg_apply_coarse_schur(wmg_ctx* ctx, int level, int prec, int dagger, const void* in_dev, void* out_dev,
                                  int nrhs);

/* ---- serving: continuous-batching solve server ----
 * Keeps several gauge fields and their hierarchies resident (one context per field, set up
 * with wmg_setup) and serves solve requests (a mass and 1..n right-hand sides) for them.
 * Each field has a worker thread and the context's own CUDA stream, so different fields'
 * work overlaps on the device.  A field's requests are batched: their right-hand sides
 * occupy the slots of one multi-right-hand-side outer solve (all slots share the field's
 * hierarchy; masses may differ, entering as diagonal shifts), and requests arriving while a
 * batch runs are admitted into slots freed by converged right-hand sides at the next restart
 * boundary.  Every right-hand side is iterated independently, so its result does not depend
 * on what else is in the batch.  Fields are admitted against an HBM budget by their
 * footprint (gauge + hierarchy + slot workspaces). */
typedef struct wmg_server wmg_server;
wmg_status wmg_server_create(wmg_server** out, size_t hbm_budget_bytes);
/* Hand a set-up context to the server (no other call may use it until wmg_server_destroy).
 * nslots (1..64): right-hand sides solved together.  WMG_ENOMEM if the budget is exceeded. */
wmg_status wmg_server_add_field(wmg_server* s, wmg_ctx* ctx, int nslots, int* field_id);
/* Queue a solve of D(m) x = b (canonical host spinors, nrhs of them).  b and x must stay valid
 * until wmg_server_wait returns for the ticket.  Thread-safe. */
wmg_status wmg_server_submit(wmg_server* s, int field_id, double mass, const double* b_host, double* x_host,
                             int nrhs, long long* ticket);
wmg_status wmg_server_poll(wmg_server* s, long long ticket, int* done);
/* Block until the request is complete; info: array of nrhs (or NULL); latency_s: seconds from
 * submission to completion (or NULL).  Returns the request's status and releases the ticket. */
wmg_status wmg_server_wait(wmg_server* s, long long ticket, wmg_info* info, double* latency_s);
/* Finish the queued work, stop the workers, free the server (the contexts stay the caller's). */
wmg_status wmg_server_destroy(wmg_server* s);

/* ---- allocation-free residual (no counterpart in the paper) ----
 * r = b - D(U) x and norm2[k] = |r_k|^2 for nrhs native fine spinors of precision prec
 * (norm2: device array of nrhs doubles, accumulated in FP64), at the context's mass.
 * For callers that must not allocate device memory inside a call: code that has handed
 * all device memory to its own arena, or code that cannot afford the device-wide
 * synchronisation a cudaMalloc / cudaFree may cause.  This call never allocates; its
 * scratch (1 MiB of partial sums, 64 counters, 64 masses) is a fixed static device array
 * that every GPU loading the library holds until exit.  Limits: nrhs <= 64 and
 * nrhs * ceil(V / 128) <= 131072 (e.g. V = 16^3 x 32 allows 64 right-hand sides,
 * V = 48^3 x 96 one); larger requests return WMG_EINVAL with the reason in
 * wmg_last_error.  The first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls
 * share the scratch: calls that overlap on the GPU race; r must not alias x.
 * Stream-ordered on the context's stream. */
wmg_status wmg_residual_noalloc(wmg_ctx* ctx, int prec, const void* b_dev, const void* x_dev, void* r_dev,
                                double* norm2_dev, int nrhs);

/* ---- instrumentation (no counterpart in the paper) ----
 * When enabled, every launch of the solver's kernels is bracketed by two CUDA events on
 * the context's stream (this adds host work per launch; leave it off for timing runs).
 * Classes: 0 sloppy fine dslash, 1 FP64 fine dslash (true residuals), 2 coarse stencil,
 * 3 restrict, 4 prolong, 5 vector updates and reductions on the fine level, 6 setup
 * (Gram-Schmidt and Galerkin construction), 7 coarsest solves run as one persistent kernel
 * (stencil applications and their vector updates together; units = right-hand sides solved),
 * 8 vector updates and reductions on the coarse levels (CG iterations, coarse smoothers).
 * wmg_profile_enable(ctx, 1) resets the counters. */
wmg_status wmg_profile_enable(wmg_ctx* ctx, int on);
/* Totals of class cls since the last enable: kernel milliseconds, launches (or launch
 * groups), the algorithmic bytes those launches must move (compulsory reads + writes:
 * operator / link / P data once, each input and output vector once per pass a kernel makes over
 * it; 0 for class 6) and the right-hand sides they processed (operator applications).
 * Synchronises. */
wmg_status wmg_profile_get(wmg_ctx* ctx, int cls, double* ms, long long* launches, double* bytes, double* units);
/* Total number of CUDA kernels this library has launched in this process (all contexts). */
wmg_status wmg_launch_count(long long* n);

/* Measured FMA throughput of the current device in TFLOP/s (2 flops per FMA), FP32 and FP64
 * (the ALU roofline denominators): dependent FMA chains over 8 CTAs of 256 threads per SM,
 * best of 3 timed launches.  Synchronises the device; takes well under a second. */
wmg_status wmg_probe_alu_peaks(double* fp32_tflops, double* fp64_tflops);

#ifdef __cplusplus
}
#endif

#endif /* WMG_H */
