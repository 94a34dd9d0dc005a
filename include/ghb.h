/*
 * ghb.h -- guaranteed homogenization bounds, Ga scheme (Galerkin approximation
 * with exact integration), GB300 (sm_103a) library.  C ABI.
 *
 * Method: J. Vondrejc, "Improved guaranteed computable bounds on homogenized
 * properties of periodic media by Fourier-Galerkin method with exact
 * integration", arXiv:1412.2033.
 *
 * Problem.  A scalar isotropic coefficient a(x) on the unit cell Y = (-1/2,1/2)^d,
 * d in {2,3}, made of a matrix value a0 and disjoint inclusions (boxes, disks,
 * spheres) -- the inclusion-matrix composite of eq. inclcomp.  For odd orders
 * N = (N_1..N_d) the library computes the Ga bounds of Def. Ga:
 *     upper U_ij = a(E_i + e_i, E_j + e_j),  e_i the minimiser over E_N (eq. GA_prim)
 *     lower L = D^{-1},  D_ij = a^{-1}(J_i + j_i, J_j + j_j), j_i over J_N
 * (Prop. struct_bounds, eq. spd_inverse_ineq), each minimiser found by conjugate
 * gradients (Remark CG) on the projected system of Cor. Ga_linsys:
 *     G A^full e = -G A^full E^,   G = G_E (primal) or G_J (dual, with 1/a).
 * The operator is applied through a double grid M >= 2N-1 (Lemma
 * integ_eval_VM, eq. MBA_GA, Algorithm 2): zero-pad Z_N -> Z_M, inverse FFT,
 * multiply by A_M(x_m) = sum_{n in Z_{2N-1}} omega_M^{mn} a^(n), forward FFT,
 * truncate to Z_N, project (Def. projection).
 *
 * Field layout (device memory, used by ghb_matvec and ghb_solve's output).
 * A trial field is a real trigonometric polynomial of Def. trig_pol, stored by
 * its Fourier coefficients as a half spectrum:
 *     x[c][i_1]...[i_{d-1}][j]      c = 0..d-1 (vector component)
 * i_a = 0..N_a-1 holds frequency k_a = i_a - (N_a-1)/2 (centred order);
 * j = 0..(N_d-1)/2 holds k_d = j (the non-negative half of the last axis).
 * Entries are complex: interleaved (re, im) pairs of double (FP64) or float
 * (FP32).  The other half is implied by Hermitian symmetry x(-k) = conj x(k);
 * on the plane k_d = 0 the caller must supply Hermitian-consistent entries.
 * Number of complex entries: d * N_1 * ... * N_{d-1} * (N_d+1)/2
 * (ghb_field_elems).
 *
 * Errors.  Every call returns a ghb_status; nothing aborts.  A failing call
 * leaves a message for ghb_last_error() (per calling thread).
 * Ownership.  Host arrays passed in are read during the call and copied;
 * device pointers passed in stay owned by the caller.  A context owns all the
 * device memory it allocates and frees it in ghb_destroy.
 * Streams.  A context issues all of its work on one CUDA stream (its own, or
 * the one given to ghb_set_stream).  ghb_solve_* and ghb_bounds return after
 * the results are on the host.  ghb_matvec is asynchronous on its stream.
 * Threads.  One context must not be used by two threads at the same time;
 * distinct contexts are independent.
 */
#ifndef GHB_H
#define GHB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ghb_ctx ghb_ctx;

typedef enum {
  GHB_OK = 0,
  GHB_ERR_INVALID = 1,        /* bad argument: even N, d not 2/3, non-positive
                                 coefficient, inclusion too large or overlapping,
                                 unsupported M, null pointer */
  GHB_ERR_OOM = 2,            /* device allocation failed */
  GHB_ERR_NOT_CONVERGED = 3,  /* max_iter reached; outputs are still filled and
                                 are still guaranteed bounds (any admissible
                                 field gives one, Prop. struct_bounds) */
  GHB_ERR_BREAKDOWN = 4,      /* CG curvature <p, Ap> not positive or not finite */
  GHB_ERR_CUDA = 5            /* a CUDA runtime call failed */
} ghb_status;

typedef enum { GHB_BOX = 0, GHB_DISK = 1, GHB_SPHERE = 2 } ghb_shape;
typedef enum {
  GHB_PRIMAL = 0,       /* Ga operator, coefficient a (eq. GA_prim) */
  GHB_DUAL = 1,         /* Ga operator, coefficient 1/a */
  GHB_GANI_PRIMAL = 2,  /* ghb_matvec only: GaNi operator (Algorithm 1), samples of a */
  GHB_GANI_DUAL = 3     /* ghb_matvec only: GaNi operator, samples of 1/a */
} ghb_kind;
typedef enum {
  GHB_FP64 = 0,   /* every operator application in FP64 */
  GHB_MIXED = 1,  /* FP32 inner CG inside an FP64 residual-correction loop; the
                     final projection and the bound energies in FP64 */
  GHB_FP32 = 2    /* ghb_matvec only: the FP32 operator */
} ghb_precision;

/* One inclusion (eq. inclcomp): characteristic function of a centred shape
 * moved to `center`, with coefficient `value` inside.
 *   GHB_BOX:    size[0..d-1] = side lengths h_a, 0 < h_a <= 1 (rect_h)
 *   GHB_DISK:   d = 2, size[0] = radius r, 0 < r <= 1/2     (circ_r)
 *   GHB_SPHERE: d = 3, size[0] = radius r, 0 < r <= 1/2
 * Fourier coefficients: Remark anal_Fourier, eq. char_func_Four; the sphere's
 * is the three-dimensional radial transform (not printed in the paper). */
typedef struct {
  int32_t shape;
  int32_t pad_;
  double center[3];
  double size[3];
  double value;
} ghb_phase;

typedef struct {
  double tol;          /* CG stop: ||r||_2 / ||b||_2 <= tol (default 1e-10) */
  int32_t max_iter;    /* per solve, counted in operator applications (default 20000) */
  int32_t precision;   /* GHB_FP64 (default) or GHB_MIXED */
  double inner_tol;    /* GHB_MIXED: relative reduction asked of each FP32 inner
                          solve (default 1e-5); a solve that needs less to
                          reach tol is asked half of what it needs (at most
                          1/2) */
  int32_t max_outer;   /* GHB_MIXED: cap on FP64 residual corrections (default 20) */
  int32_t M[3];        /* double grid per axis; 0 = automatic: the smallest
                          M_a >= 2 N_a - 1 whose prime factors are 2, 3, 5.
                          Any M_a >= 2 N_a - 1 whose prime factors are <= 31
                          is accepted (Lemma integ_eval_VM: the bilinear form
                          does not depend on M). */
} ghb_options;

typedef struct {
  int32_t status;        /* ghb_status of this solve */
  int32_t iters;         /* CG iterations (all inner iterations for GHB_MIXED) */
  int32_t outer_iters;   /* FP64 residual corrections (GHB_MIXED), else 0 */
  int32_t matvecs_fp64;  /* FP64 operator applications */
  int32_t matvecs_fp32;  /* FP32 operator applications */
  int32_t pad_;
  double relres;         /* final ||r||/||b|| of the FP64 system */
  double energy;         /* a(E+e, E+e) (primal) or a^{-1}(J+j, J+j) (dual), FP64 */
} ghb_solve_info;

/* Form of the Ga operator (the same operator, Lemma reduce_grid):
 *   GHB_FORM_DOUBLE_GRID  Algorithm 2: one transform of length M per axis and
 *                         line (the default);
 *   GHB_FORM_REDUCED      Algorithm 3: for every s in {0,1}^d the N-length
 *                         transforms of the field shifted by S(s) =
 *                         diag(omega_2N^{-s.m}), multiplied by the double-grid
 *                         values at the points 2r - s; needs M = 2N on every
 *                         axis; N-sized intermediates. */
typedef enum { GHB_FORM_DOUBLE_GRID = 0, GHB_FORM_REDUCED = 1 } ghb_form;

/* Default options (tol 1e-10, FP64, automatic M). */
void ghb_default_options(ghb_options* opt);

/* Create a context for dimension d, odd orders N[0..d-1], matrix value a0 and
 * n_phases inclusions.  Builds, on the device, the coefficient tables a^ and
 * (1/a)^ on Z_{2N-1} (eq. inclcomp_formula) and their double-grid values A_M,
 * B_M (eq. MBA_GA).  `opt` may be NULL for defaults.  On success *out owns the
 * context; on failure *out is NULL. */
ghb_status ghb_create(ghb_ctx** out, int d, const int* N, double a0,
                      const ghb_phase* phases, int n_phases, const ghb_options* opt);

/* Grid-based composite (Lemma grid_compos, Remark eval_with_FFT): a(x) is the
 * piecewise-constant pixel (voxel) image with image[p] on the pixel of side
 * 1/P_a centred at x = p / P (periodic), p_a = 0 .. P_a - 1, C-order, host
 * memory, every value positive and finite; P_a in 1..8192 with prime factors
 * <= 31 (any relation to N is allowed: the image's spectrum is truncated or
 * periodically extended to Z_{2N-1}).  The tables are a^(m) = prod_a
 * sinc(m_a / P_a) (1/|P|) sum_p image[p] w_P^{-m.p} and the same for 1/image
 * (the inverse of a pixel image is the pixel image of the inverses); the
 * double-grid values follow as for inclusions.  Every solve and bound call
 * then applies to the image; ghb_bounds_gani is not available (GHB_ERR_INVALID).
 * ghb_set_image replaces the coefficients of an existing context (any
 * resolution P); ghb_set_coeffs switches back to inclusions. */
ghb_status ghb_create_image(ghb_ctx** out, int d, const int* N, const int* P, const double* image,
                            const ghb_options* opt);
ghb_status ghb_set_image(ghb_ctx* ctx, const int* P, const double* image);

/* Replace the microstructure (same d, N, M): rebuild a^, (1/a)^, A_M, B_M. */
ghb_status ghb_set_coeffs(ghb_ctx* ctx, double a0, const ghb_phase* phases, int n_phases);

/* Select the form of the Ga operator used by ghb_matvec (Ga kinds), the solves
 * and the bounds (the Gram energies are always evaluated on the double grid).
 * GHB_ERR_INVALID if the form is unknown, or GHB_FORM_REDUCED with M != 2N or
 * with an N that has a prime factor above 31.  The sub-grids of the reduced
 * form follow later coefficient changes. */
ghb_status ghb_set_form(ghb_ctx* ctx, int form);

/* Replace the options of an existing context (M is fixed at creation and ignored). */
ghb_status ghb_set_options(ghb_ctx* ctx, const ghb_options* opt);

/* Use `stream` (a cudaStream_t, or NULL for the context's own) for all work. */
ghb_status ghb_set_stream(ghb_ctx* ctx, void* stream);

/* Grid sizes: N_out[0..d-1], M_out[0..d-1] (may be NULL) and the number of
 * complex entries of one field in the half-spectrum layout above. */
ghb_status ghb_get_grid(const ghb_ctx* ctx, int* d_out, int* N_out, int* M_out,
                        int64_t* field_elems);
int64_t ghb_field_elems(const ghb_ctx* ctx);

/* y = G A^full x (kind = GHB_PRIMAL: G_E and a; GHB_DUAL: G_J and 1/a; the
 * GaNi operator G a~_N of Algorithm 1 for GHB_GANI_PRIMAL / GHB_GANI_DUAL) for one
 * field in the half-spectrum layout; precision GHB_FP64 (double pairs) or
 * GHB_FP32 (float pairs).  x_dev, y_dev: device pointers, caller-owned, not
 * overlapping.  project = 0 skips G (returns A^full x, used for energies).
 * Asynchronous on `stream` (NULL = the context's stream). */
ghb_status ghb_matvec(ghb_ctx* ctx, int kind, int precision, int project,
                      const void* x_dev, void* y_dev, void* stream);

/* Minimise a(E + e, E + e) over e in E_N (primal) or a^{-1}(J + j, J + j)
 * over j in J_N (dual) for the load E[0..d-1].  If field_out_dev is not NULL
 * the admissible field E + e (FP64 half spectrum) is written there.  `info`
 * (may be NULL) receives iterations, residual and the FP64 energy. */
ghb_status ghb_solve_primal(ghb_ctx* ctx, const double* E, void* field_out_dev,
                            ghb_solve_info* info);
ghb_status ghb_solve_dual(ghb_ctx* ctx, const double* J, void* field_out_dev,
                          ghb_solve_info* info);

/* One solve with an initial guess and bound tracking (Section 7.4, the
 * evolution of the bounds during CG, and the coarse-to-fine start).
 *   kind: GHB_PRIMAL or GHB_DUAL; E[d]: load; field_out_dev, info: as for
 *     ghb_solve_primal (info->energy is the exact energy of the final field);
 *   x0_dev: initial fluctuation e_0, FP64 half spectrum of this context's N,
 *     admissible (in the range of the projection, e.g. a prolongated coarse
 *     solution minus its load); NULL = 0, the start at the Voigt (Reuss) value;
 *   energies (host, may be NULL), cap >= 1: the energy a(E + e_i, E + e_i)
 *     (primal; a^{-1}(.,.) dual) along the iterates, an upper bound (primal) or
 *     the inverse of a lower bound (dual) at every step.  FP64 precision: one
 *     value per CG iterate from the CG scalars, J(e_i) = J(e_0) -
 *     sum_{j<i} alpha_j <r_j, r_j>, with J(e_0) evaluated exactly; mixed: the
 *     start and every FP64 correction, each an exact Gram evaluation.
 *     *n_energies (may be NULL) receives the count (at most cap).
 * Returns the solve's status (GHB_ERR_NOT_CONVERGED keeps the outputs). */
ghb_status ghb_solve_ex(ghb_ctx* ctx, int kind, const double* E, const void* x0_dev, void* field_out_dev,
                        ghb_solve_info* info, double* energies, int cap, int* n_energies);

/* Prolongation I_Nf o I_Nc^{-1} (Section 7.4): writes to xf_dev (Z_Nf) the
 * coefficients of the same trigonometric polynomial as xc_dev (Z_Nc), zero at
 * the frequencies outside Z_Nc; no approximation is made.  d fields of FP64
 * half spectra (layout above), orders odd with Nf_a >= Nc_a.  Synchronous on
 * `stream` (NULL = legacy default stream). */
ghb_status ghb_prolong(int d, const int* Nc, const void* xc_dev, const int* Nf, void* xf_dev, void* stream);

/* The Gram matrix out[i*m + j] = a(v_i, v_j) (kind primal) or a^{-1}(v_i, v_j)
 * (dual) of m <= 3 FP64 fields v_i given as device pointers, evaluated exactly
 * on the double grid in FP64 (Lemma integ_eval_VM): (1/|M|) sum_m A_M(x_m)
 * v_i(x_m).v_j(x_m).  Synchronous. */
ghb_status ghb_gram(ghb_ctx* ctx, int kind, int m, const void* const* fields_dev,
                    double* out);

/* Both bounds: d primal and d dual solves with unit loads, then the Gram
 * matrices; upper[d*d] = U, lower[d*d] = D^{-1} (row-major, symmetrised).
 * infos (may be NULL) receives 2d entries: primal e_1..e_d, dual e_1..e_d. */
ghb_status ghb_bounds(ghb_ctx* ctx, double* upper, double* lower, ghb_solve_info* infos);

/* GaNi scheme (Def. GaNi, Algorithm 1) and its a-posteriori guaranteed bounds
 * (eq. GaNi_apost).  The minimisers e~_i (primal) and j~_i (dual) of the
 * trapezoidal-rule energies (1/|N|) sum_k a(x^k) v(x^k).v(x^k), x^k = k/N (a
 * point on an inclusion's boundary counts as inside), are found by CG with the
 * context's precision on the N grid; then
 *   upper[d*d]      = a(E_i + e~_i, E_j + e~_j), the exact energies on the
 *                     double grid (a guaranteed upper bound),
 *   lower[d*d]      = inverse of a^{-1}(J_i + j~_i, J_j + j~_j) (guaranteed lower),
 *   a_gani[d*d]     = the GaNi matrix A~_N (trapezoidal energies; may be NULL),
 *   b_gani_inv[d*d] = B~_N^{-1} (may be NULL; equals A~_N for odd N, Remark
 *                     duality_gani);
 * row-major, symmetrised.  Every transform length N_a must have prime factors
 * <= 31 (else GHB_ERR_INVALID).  infos as for ghb_bounds (energy = exact).
 * The Ga bounds of ghb_bounds lie inside [lower, upper] (Ga minimises the exact
 * energy over the same space).  Synchronous. */
ghb_status ghb_bounds_gani(ghb_ctx* ctx, double* upper, double* lower, double* a_gani, double* b_gani_inv,
                           ghb_solve_info* infos);

/* Device data for checks: the coefficient table a^ (kind primal) or (1/a)^
 * (dual) on Z_{2N-1} as a half spectrum (centred leading axes of length
 * 2N_a-1, last axis n_d = 0..N_d-1; complex FP64), or the double-grid values
 * A_M / B_M (real FP64, C-order over m_a = 0..M_a-1, grid point x = m/M).
 * `out_dev` must hold the stated number of entries (ghb_table_elems /
 * ghb_grid_elems).  Synchronous. */
int64_t ghb_table_elems(const ghb_ctx* ctx);
int64_t ghb_grid_elems(const ghb_ctx* ctx);
ghb_status ghb_copy_table(ghb_ctx* ctx, int kind, void* out_dev);
ghb_status ghb_copy_grid_values(ghb_ctx* ctx, int kind, void* out_dev);

/* Timing of the context's own launches.  ghb_profile(ctx, 1) starts recording a
 * pair of CUDA events around every kernel launch on the context's stream
 * (launches queued after a CG solve ended are dropped), ghb_profile(ctx, 0)
 * stops; both clear earlier records.  ghb_profile_read sums the records of one
 * kernel class: cls = 2 * k + f, f = 1 for the FP32 variant, k one of
 *   0 coefficient set-up, 1 axis-1 inverse pass fused with the CG direction
 *   update, 2 axis-1 inverse pass, 3 axis-2 inverse pass, 4 last-axis pass
 *   (inverse, multiply by A_M, forward), 5 axis-2 forward pass, 6 axis-1
 *   forward pass with truncation, 7 projection + <p, Ap>, 8 CG vector update
 *   + <r, r>, 9 projection, 10 FP64 residual, 11 Gram pass, 12 other.
 * It returns the number of launches, their summed duration in ms, and the
 * algorithmic bytes and FFT flops (5 L log2 L per length-L complex transform)
 * of one launch of that class for this context's sizes. */
ghb_status ghb_profile(ghb_ctx* ctx, int enable);
ghb_status ghb_profile_read(ghb_ctx* ctx, int cls, int64_t* launches, double* total_ms,
                            double* bytes_per_launch, double* flops_per_launch);

/* ------------------------------------------------------------------------
 * Batched and served solving.  A batch holds many bound-pair requests (each
 * one microstructure at its own d and N) and solves them together in the
 * mixed scheme: every CG iteration is one launch per kernel over all active
 * solves, whatever their sizes.  Requests are admitted while their device
 * memory (coefficient grids, CG vectors, intermediates of their 2d solves)
 * fits the batch's budget, so requests submitted while others run join the
 * running work at the next step (continuous batching); finished requests leave
 * and free their memory.  A batch owns its CUDA stream and device memory.
 * Requests of at least 2^22 double-grid points (d = 3 from M = 162, d = 2 from
 * M = 2048) are solved instead by two worker threads of the batch, each with a
 * private context on its own stream, while the batched cycles run (a
 * large solve would otherwise set the pace of every batched iteration); their
 * results enter the same queue, and the context's memory counts against the
 * budget while it exists.
 * ------------------------------------------------------------------------ */
typedef struct ghb_batch ghb_batch;

typedef struct {
  int64_t id;              /* as returned by ghb_batch_submit */
  int32_t d;
  int32_t status;          /* ghb_status of the request */
  double upper[9];         /* d x d row-major */
  double lower[9];
  ghb_solve_info info[6];  /* primal e_1..e_d, then dual e_1..e_d */
  double seconds_queued;   /* submission -> admission (host clock) */
  double seconds_total;    /* submission -> result */
} ghb_result;

/* Create a batch.  opt: NULL for defaults (precision must be GHB_MIXED);
 * budget_bytes: device-memory budget for admitted requests (0 = 60% of the
 * free memory now); max_active: cap on requests solved at once (0 = 4096). */
ghb_status ghb_batch_create(ghb_batch** out, const ghb_options* opt, int64_t budget_bytes, int max_active);

/* Queue one bound-pair request (same microstructure description and checks as
 * ghb_create).  Host arrays are copied.  *id_out receives its id. */
ghb_status ghb_batch_submit(ghb_batch* b, int d, const int* N, double a0, const ghb_phase* phases,
                            int n_phases, int64_t* id_out);

/* One engine cycle: admit pending requests that fit, run `iterations` batched
 * FP32 CG iterations (0 = 8) over all active solves, apply the FP64
 * corrections of solves whose inner CG ended, and finish the requests whose
 * solves all ended.  Synchronises with the device.  *active_out, *pending_out
 * (may be NULL) receive the counts after the cycle. */
ghb_status ghb_batch_step(ghb_batch* b, int iterations, int* active_out, int* pending_out);

/* Step until every submitted request has finished. */
ghb_status ghb_batch_run(ghb_batch* b, int iterations);

/* Move up to max_results finished results into out[]; returns how many. */
int ghb_batch_results(ghb_batch* b, ghb_result* out, int max_results);

ghb_status ghb_batch_stats(const ghb_batch* b, int64_t* bytes_in_use, int* active, int* pending,
                           int64_t* finished, int64_t* launches);

/* Release the batch (pending and running requests are dropped; large requests
 * in progress in the workers finish first).  NULL is a no-op. */
void ghb_batch_destroy(ghb_batch* b);

/* ghb_gram without any device allocation (the paper has no counterpart; this
 * is a library convenience).  For callers that cannot call cudaMalloc: code
 * running inside another framework's memory arena that must not grow the
 * device heap behind its back, code running with device memory reserved to
 * the last byte, or code under a no-allocation-after-start-up policy.
 *   d, N[d], M[d]: dimension, odd orders, double grid (M_a >= 2N_a - 1, prime
 *     factors <= 31), as for a context;
 *   grid_dev: the double-grid values A_M (or B_M), FP64, C-order over
 *     m_a = 0..M_a-1 (for example from ghb_copy_grid_values);
 *   fields_dev[0..m-1], 1 <= m <= d: FP64 half-spectrum fields (layout above);
 *   out[m*m]: host, receives a(v_i, v_j) = (1/|M|) sum_m A_M(x_m) v_i.v_j;
 *   stream: cudaStream_t or NULL (legacy default stream).  Synchronous.
 * All scratch (transform tables, intermediates, partial sums) lives in one
 * fixed 32 MiB device array that every GPU loading this library holds until
 * the process exits; sizes needing more are rejected with GHB_ERR_INVALID
 * and a message (d = 2 reaches N = 511 for m = 2).  The call allocates
 * nothing (no cudaMalloc, cudaFree, or allocating library routine).  The
 * first call on a device looks up the array's device address on that device,
 * so make it before any stream capture.  Every call shares the one array and
 * leaves its contents behind: calls that overlap on the GPU (other streams or
 * host threads) race and must be serialised by the caller. */
ghb_status ghb_gram_noalloc(int d, const int* N, const int* M, const double* grid_dev, int m,
                            const void* const* fields_dev, double* out, void* stream);

/* ---------------------------------------------------------------------------
 * Launch configuration of the transform passes (no counterpart in the paper:
 * it decides how the FFTs of Algorithm 2 are laid out on the GPU, not what
 * they compute).  Per transform length M the library holds
 *   cfg[0] cap32   largest radix product of one register-blocked pass of the
 *                  runtime-plan FP32 transform (5..32)
 *   cfg[1] tile32  columns per CTA of the FP32 column passes (0 = chosen at
 *                  each launch from the operand's shape: the widest tile whose
 *                  CTAs fill the device three times over; else 1, 2, 4, 8 or 16
 *                  within shared memory, forced)
 *   cfg[2] rows32  rows per CTA of the FP32 2-D last-axis pass (0 = size rule,
 *                  1 or 2)
 *   cfg[3] ct_col  1: size-specialised FP32 column kernels (only for lengths
 *                  that have them: 72, 135, 162, 270, 486, 1458, 2187,
 *                  4374), 0: runtime plan
 *   cfg[4] ct_row  the same for the last-axis pass
 *   cfg[5] cap64   as cap32 for FP64
 *   cfg[6] tile64  as tile32 for FP64
 * The first plan for M in a process times the candidates for cfg[0], [2], [3],
 * [4] and [5] on a 2-D operand of at least 2^20 double-grid entries with CUDA
 * events and keeps the fastest (the autotuner; the tiles stay 0); setting the
 * environment variable GHB_AUTOTUNE=0 keeps the size rules instead.  Every
 * configuration computes the same operator; results differ only by rounding.
 * A configuration applies to plans made after it is fixed (contexts and batch
 * instances created later).
 *
 * ghb_tune_get: cfg[7] host, receives M's configuration, tuning M first if it
 *   has not been (this allocates and runs kernels on the current device).
 * ghb_tune_set: fixes M's configuration to cfg[7] (validated; GHB_ERR_INVALID
 *   with a message otherwise).
 * ghb_tune_reset: forgets every stored configuration.
 * All three are thread-safe; M must factor into primes <= 31. */
ghb_status ghb_tune_get(int M, int* cfg);
ghb_status ghb_tune_set(int M, const int* cfg);
ghb_status ghb_tune_reset(void);

/* Device bytes held by the context. */
int64_t ghb_device_bytes(const ghb_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* ghb_last_error(void);

/* Release the context and all device memory it owns.  NULL is a no-op. */
void ghb_destroy(ghb_ctx* ctx);

/* Library version string. */
const char* ghb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GHB_H */
