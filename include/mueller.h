/*
 * mueller.h -- C ABI of the GB300 separation-of-variables Mueller solver for
 * penetrable bodies of revolution (Lai & O'Neil, arXiv:1810.07067).
 *
 * The body is the rotation of a generating curve gamma(s) = (r(s), z(s)) about
 * the z axis (Section 3).  The curve is given as panels of p = 16 nodes placed
 * at the Gauss-Legendre points of a panel-local parameter tau in [-1, 1]
 * (Section 5).  For every Fourier mode m the solver assembles the dense
 * 4N x 4N Nystrom system of the Mueller integral equation (eq. mullerrep, or
 * its indirect form eq. dualmullrep), factors it by LU with partial pivoting
 * and solves for the modal currents (J^1_m, J^2_m, M^1_m, M^2_m) at each node
 * (J = J^1 t + J^2 e_theta, M likewise; Section 3).
 *
 * Conventions used by every entry point
 *  - Complex numbers are mueller_c128 {re, im} (binary compatible with a
 *    C99 double complex, std::complex<double> and torch.complex128).
 *  - "host" pointers are ordinary CPU memory read during the call; "device"
 *    pointers are CUDA global memory of the current device, owned by the
 *    caller, read or written asynchronously on the given CUDA stream
 *    (cudaStream_t passed as void*; NULL = legacy default stream).
 *  - Node n of the curve owns unknowns 4n+0 (J^1), 4n+1 (J^2), 4n+2 (M^1),
 *    4n+3 (M^2) and equations 4n+0 (E_t), 4n+1 (E_theta), 4n+2 (H_t),
 *    4n+3 (H_theta).  Modal vectors are stored [2M+1][nrhs][4N] with mode
 *    index q = m + M.
 *  - Every call returns a mueller_status; nothing is thrown across the ABI.
 *    No entry point falls back to a CPU implementation.
 */
#ifndef MUELLER_H
#define MUELLER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } mueller_c128;
typedef struct { float re, im; } mueller_c64;

typedef enum {
  MUELLER_OK = 0,
  MUELLER_EINVAL = 1,     /* invalid argument (message via mueller_last_error) */
  MUELLER_ENOMEM = 2,     /* device or host allocation failed                  */
  MUELLER_ESINGULAR = 3,  /* exact zero pivot in some mode (see stats)         */
  MUELLER_ENOCONV = 4,    /* iterative refinement hit its cap                  */
  MUELLER_ETIMEOUT = 5,   /* a bounded device-side wait gave up (for tests,
                             the environment variable MUELLER_FAULT_INJECT =
                             "lu_timeout" and/or "residual_timeout" makes the
                             host set that status word before reading it, so
                             the error path runs without a device fault)     */
  MUELLER_ECUDA = 6       /* CUDA runtime error                                */
} mueller_status;

/* Generating curve (host arrays, copied during the call).
 * Nodes are panel-major: node n = 16*panel + local index, local index k at
 * tau_k, the k-th 16-point Gauss-Legendre node of [-1, 1] in increasing
 * order.  The curve runs counterclockwise in the (r, z) half plane, so that
 * n = (z', -r') points out of the body (Section 3); open curves start and end
 * on the axis.  dr, dz are derivatives with respect to tau (the parameter
 * need not be arclength; Section 6).  Geometry between nodes (support points
 * of the near-panel rules) is the degree-15 Lagrange interpolant of the node
 * values of r, z, dr, dz on the panel. */
typedef struct {
  int n_panels;        /* >= 1; N = 16 * n_panels nodes                   */
  int closed;          /* 1: first and last panel are neighbours (torus)  */
  const double* r;     /* [N] host, r > 0                                  */
  const double* z;     /* [N] host                                         */
  const double* dr;    /* [N] host, dr/dtau                                */
  const double* dz;    /* [N] host, dz/dtau                                */
} mueller_curve;

/* Media (Section 1, eq. materials): background (0) and body (1);
 * k_j = omega * sqrt(eps_j mu_j) (principal root).  Requires omega > 0,
 * Re eps_j, Re mu_j > 0 and Im eps_j, Im mu_j >= 0. */
typedef struct {
  double omega;
  mueller_c128 eps0, mu0, eps1, mu1;
} mueller_media;

typedef struct {
  int n_phi;           /* azimuthal samples (power of two >= 16); raised
                          automatically when too small for M and k (see
                          stats.n_phi_used).  One warp's shared memory,
                          80 n_phi + 144 M + 440 bytes, must fit the device's
                          opt-in limit per CTA (232,448 bytes on GB300, e.g.
                          n_phi = 2048 with M <= 473); larger requests fail
                          with MUELLER_EINVAL before any device work         */
  int formulation;     /* 0 direct (eq. mullerrep), 1 indirect (eq. dualmullrep) */
  int precision;       /* 0 FP64; 1 mixed: complex64 LU + iterative refinement
                          whose complex128-accurate residuals run on BF16
                          tensor cores (exact 8-digit slicing of A' and y);
                          2 mixed with residuals on the FP64 pipe           */
  double refine_tol;   /* mixed: stop when backward error <= refine_tol     */
  int refine_max_iter; /* mixed: cap on refinement steps                    */
  double split_eps;    /* kernel splitting when the plain trapezoid would
                          alias above this (default 1e-17 when <= 0)         */
  int lu_tile;         /* mixed path: column tile of the tensor-core LU update,
                          32, 64 or 128; 0 = chosen per step by the tile
                          autotuner (timed once per process for each bucket
                          of trailing size and matrix count, see
                          mueller_lu_tile_table)                            */
} mueller_options;

typedef struct {
  double ms_legendre, ms_far, ms_support, ms_near, ms_lu, ms_build;  /* stage times; ms_lu is the
                                factorization alone, ms_build assembly (with the mixed path's
                                complex64 copy and digit slices) plus ms_lu */
  double ms_solve;           /* last mueller_solve                           */
  int n_phi_used;
  long long n_split_pairs;   /* pairs evaluated with kernel splitting        */
  long long n_far_pairs, n_support_pairs;
  int singular_mode;         /* first mode with a zero pivot, or -1          */
  int singular_column;
  size_t device_bytes;       /* memory held by the context                   */
  double ms_lu_gemm;         /* device time of the LU trailing-update launches */
  double lu_gemm_flops;      /* their algorithmic flops (8 per complex FMA)  */
  int lu_gemm_launches;
  int launches;              /* kernel launches of the last build            */
  int solve_launches;        /* kernel launches of the last solve            */
  int refine_iters;          /* mixed path: refinement steps of the last solve */
  double backward_err_max;   /* mixed path: largest final backward error       */
  double ms_residual;        /* precision 1: device time of the tensor-core residuals (incl. slicing) */
  int residual_launches;     /* precision 1: residual evaluations of the last solve */
  double residual_tc_flops;  /* precision 1: their BF16 tensor work (2 flops per MAC) */
  int lu_graph;              /* 1: the LU steps ran as one captured CUDA graph */
  int lu_tile_steps[3];      /* mixed path: LU steps whose update used column tiles 32, 64, 128 */
  int lu_wave_bodies;        /* bodies factored together (mueller_build_many), else 1 */
  int lu_launches;           /* kernel launches (graph nodes) of the factorization, shared by a wave */
  double lu_gemm_bytes;      /* bytes of the trailing matrices the updates read and write (once each) */
  int spilled;               /* 1 while the device buffers are in host memory (mueller_ctx_spill) */
  size_t host_bytes;         /* pinned host bytes held while spilled */
  double kappa_mode0;        /* last mueller_cond_estimate: kappa_inf of mode 0 ...   */
  double kappa_max;          /* ... the largest over modes 0..M ...                   */
  int kappa_max_mode;        /* ... and its mode (-1 before any estimate)             */
  double ms_cond;            /* device time of that estimate                          */
  double ms_far_sample;      /* far pairs on the tensor-core path (0 otherwise): device time of the sampling */
  double ms_far_product;     /* ... of the digit products (the transform) ...                                */
  double ms_far_assemble;    /* ... and of the block assembly (all within ms_far)                            */
  double far_blocks;         /* 4 x 4 blocks the far-pair assembly formed (pairs x modes up to m_c + 1)       */
} mueller_stats;

typedef struct mueller_ctx mueller_ctx;

/* Build: assemble the per-mode systems for modes m = 0..M on the device and
 * factor them by LU with partial pivoting (Sections 3-5; eq. mullerrep or
 * eq. dualmullrep; "LU-factorization" of Section 6).  Modes -M..-1 are not
 * assembled: the reflection theta -> -theta gives A_{-m} = D_r A_m D_c with
 * D_r = diag(-1, 1, 1, -1) and D_c = diag(1, -1, -1, 1) per node, and
 * mueller_solve uses the factors of A_m for both.  Rows and unknowns are
 * L2-weighted internally (Section 6 remark); the API stays in physical
 * unknowns.  Host inputs are copied; the context owns all device memory of
 * the body.  Besides it the library keeps, per device and until exit, the
 * BF16 digits of the cosine matrices of the transform over phi, one per grid
 * size and mode count in use (about 21 MB for every grid up to n_phi = 512 at
 * M = 128), built on the host by the first build that needs them (which then
 * waits once for their upload on `stream`).  Work runs on `stream`; the call
 * returns after the factorization has finished (stage times are measured
 * with CUDA events). */
int mueller_build(const mueller_curve* curve, const mueller_media* media, int M,
                  const mueller_options* opts, void* stream, mueller_ctx** out);

/* Build a wave of bodies (Section 6's per-mode factorizations for several
 * bodies at once): each body i (curves[i], media[i], modes 0..M[i], all with
 * the same opts) is assembled in turn as in mueller_build; then the LU
 * factorizations of all modes of all bodies run together, one launch per
 * kernel and LU step over every (body, mode) matrix of any size, largest
 * first, the whole step sequence captured into one CUDA graph and launched
 * once on `stream`.  out[i] receives body i's context (the same factors a
 * separate mueller_build gives with the same lu_tile); on failure every out[i]
 * is NULL, except MUELLER_ESINGULAR, where all contexts are returned and the
 * singular body's stats name the mode.  Stage times of each body: its own
 * assembly; ms_lu is the wave's factorization.  At most 65535 mode matrices
 * per wave.  Device memory: mueller_build_many_bytes. */
int mueller_build_many(int count, const mueller_curve* curves, const mueller_media* media, const int* M,
                       const mueller_options* opts, void* stream, mueller_ctx** out);

/* Assemble only (no factorization) into a caller buffer A_dev
 * [M+1][4N][4N] column-major per mode, L2-weighted:
 * A'_m = diag(sqrt w) A_m diag(1/sqrt w), w the ds-weights of the nodes. */
int mueller_assemble(const mueller_curve* curve, const mueller_media* media, int M,
                     const mueller_options* opts, mueller_c128* A_dev, void* stream);

/* Solve for all modes -M..M (Section 6, T_add: additional right-hand sides
 * reuse the factors).  rhs_dev and x_dev are device arrays
 * [2M+1][nrhs][4N]; backward_err (host, [2M+1][nrhs]) may be NULL.
 * FP64 path: one solve with the complex128 factors (backward_err = -1, not
 * computed).  Mixed path: y0 from the complex64 factors, then
 * y <- y + LU32^{-1}(b' - A' y) with complex128 residuals of the L2-weighted
 * matrices until ||b' - A'y||_inf <= refine_tol (||A'||_inf ||y||_inf + ||b'||_inf)
 * for every mode and right-hand side (the normwise backward errors are
 * returned); MUELLER_ENOCONV with the last iterate if refine_max_iter steps
 * do not reach it. */
int mueller_solve(mueller_ctx* ctx, const mueller_c128* rhs_dev, int nrhs, mueller_c128* x_dev,
                  double* backward_err, void* stream);

/* Modal right-hand sides of plane waves (eq. pw): E = e exp(i k0 d.x),
 * H = (k0/(omega mu0)) d x e exp(i k0 d.x); dirs and pols are host [nrhs][3]
 * (pols = unit e, orthogonal to d).  Rows are the Fourier coefficients
 * (1/2pi) int f e^{-i m theta} of the tangential traces n x E and n x H, scaled
 * by i omega eps0 and i omega mu0 (eq. mullerrep) or i omega mu0 and
 * i omega eps0 (eq. dualmullrep).  rhs_dev: [2M+1][nrhs][4N]. */
int mueller_rhs_planewave(mueller_ctx* ctx, const double* dirs, const double* pols, int nrhs,
                          mueller_c128* rhs_dev, void* stream);

/* Modal right-hand sides from incident fields sampled by the caller (for
 * fields other than plane waves, e.g. the current loop of Section 6,
 * eq. loop).  EH_dev: device [nrhs][N][n_theta][6] complex, (E, H) in
 * Cartesian components at the ring points (r_i cos th, r_i sin th, z_i),
 * th = 2 pi t / n_theta, nodes in curve order; 2M+2 <= n_theta <= 2048.
 * Traces, Fourier coefficients and row scaling as mueller_rhs_planewave;
 * rhs_dev: [2M+1][nrhs][4N]. */
int mueller_rhs_fields(mueller_ctx* ctx, const mueller_c128* EH_dev, int nrhs, int n_theta,
                       mueller_c128* rhs_dev, void* stream);

/* Far field of mueller_far_field on the grid theta_p = (p + 1/2) pi / n_polar
 * (p < n_polar), phi_s = 2 pi s / n_azim (s < n_azim <= 8192), computed by
 * modes: for each theta, the ring integrals become per-mode coefficients and
 * the far field is a sum over m of e^{i m phi} times a per-mode vector
 * (Section 4's separation of variables applied to eq. farfieldform), then
 * rotated to Cartesian components.  x_dev: currents [2M+1][nrhs][4N];
 * E_dev: device [nrhs][n_polar][n_azim][3]. */
int mueller_far_field_grid(mueller_ctx* ctx, const mueller_c128* x_dev, int nrhs, int n_polar, int n_azim,
                           mueller_c128* E_dev, void* stream);

/* Fields at points off the surface from modal currents (Section 3):
 * region 0 (the exterior medium) by eq. exteriorfield with k0; region 1 (the
 * body) by eq. interiorfield for the direct formulation or eq. interior_dual
 * for the indirect one, with k1.  The surface integrals are refined for the
 * closest targets: each panel is split into up to 16 sub-panels of 16 Gauss
 * points (more the closer a target is relative to the panel's length), with
 * geometry and currents from the panel's degree-15 interpolants, and the
 * azimuthal trapezoid rule has max(2M + 2 ceil(|k| r_max) + 64,
 * 40 r_max / d_min) points (at most 8192), d_min the closest target-to-node
 * distance.  A target on a node ring is rejected (MUELLER_EINVAL).  x_dev:
 * currents [2M+1][nrhs][4N]; targets: host [ntargets][3]; out_dev: device
 * [nrhs][ntargets][6] complex, (E, H) in Cartesian components. */
int mueller_eval(mueller_ctx* ctx, const mueller_c128* x_dev, int nrhs, const double* targets, int ntargets,
                 int region, mueller_c128* out_dev, void* stream);

/* Far field (eq. farfieldform, with the magnetic current in the last term as
 * in eq. exteriorfield): E_oo(xh) = (1/4pi)[-(k0^2/(i omega eps0))(Jh - (xh.Jh)xh)
 * + i k0 xh x Mh], Jh = int exp(-i k0 xh.y) J(y) da(y).  x_dev: currents
 * [2M+1][nrhs][4N]; dirs_dev: device [ndir][3] unit vectors; E_dev: device
 * [nrhs][ndir][3]. */
int mueller_far_field(mueller_ctx* ctx, const mueller_c128* x_dev, int nrhs, const double* dirs_dev,
                      int ndir, mueller_c128* E_dev, void* stream);

/* Modal Green's function spectra for arbitrary (target, source) pairs
 * (Section 4): pairs_host [npairs][4] = (r_t, z_t, r_s, z_s); out_dev
 * [npairs][9][M+2] for m = 0..M+1 of: g^{k0}, g^{k1} (eq. green11),
 * d/dr_t and d/dz_t of g^{k0} and of g^{k1} (eq. firstder), and
 * d2/dr_t2, d2/dr_t dz_t, d2/dz_t2 of g^{k0} - g^{k1} (Section 4.3),
 * each the integral over phi in [0, 2pi) of the kernel times cos(m phi).
 * k0, k1 with Im >= 0; n_phi as in mueller_options. */
int mueller_modal_kernels(const double* pairs_host, long long npairs, mueller_c128 k0, mueller_c128 k1,
                          int M, int n_phi, double split_eps, mueller_c128* out_dev, void* stream);

/* Allocation-free variant of mueller_modal_kernels.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory,
 * for example a host application whose device memory is owned by another
 * allocator (a framework's memory pool, or a budget enforced by a serving
 * runtime), or a latency-critical loop in which a cudaMalloc could block or
 * fail.  It computes the same spectra as mueller_modal_kernels, but
 *  - pairs_dev is a DEVICE array [npairs][4] = (r_t, z_t, r_s, z_s), with
 *    r_t, r_s > 0 and distinct points (not checked on the host; a bad pair
 *    yields non-finite values in its own output rows);
 *  - n_phi is used as given (power of two in [16, 8192], >= 2M + 4, and
 *    within the shared-memory bound stated at mueller_options.n_phi); unlike
 *    mueller_modal_kernels it is not raised automatically, so the caller
 *    picks it large enough for the wavenumbers (see stats.n_phi_used of a
 *    build for a safe value);
 *  - all scratch (transform tables, split flags, pair displacements and
 *    Laplace-type coefficients) lives in one fixed 16 MiB device array that
 *    every GPU loading the library holds until the process exits; a call is
 *    rejected with MUELLER_EINVAL when
 *    n_phi + npairs * (n_phi/2 + M + 7) (rounded up) exceeds 2^21 doubles;
 *  - it calls no cudaMalloc, cudaFree or allocating library routine.
 * The first call on a device performs a one-time set-up on that device (it
 * looks up the scratch array's device address and uploads series tables);
 * make that first call before any stream capture.  All calls share the one
 * array and every call rewrites the parts it reads, so no state carries over,
 * but calls that overlap on the GPU (several streams, threads or processes
 * using the same device) race on the scratch and must be serialised by the
 * caller.  The work is enqueued on `stream`; the call does not synchronise. */
int mueller_modal_kernels_noalloc(const double* pairs_dev, long long npairs, mueller_c128 k0, mueller_c128 k1,
                                  int M, int n_phi, double split_eps, mueller_c128* out_dev, void* stream);

/* Batched LU of `batch` column-major n x n complex matrices in place
 * (stride n*n); piv_dev [batch][n] (0-based LAPACK-style interchanges),
 * info_dev [batch] (0 or first zero-pivot column + 1). */
int mueller_lu_batched(mueller_c128* A_dev, int n, int batch, int* piv_dev, int* info_dev, void* stream);

/* The same factorisation in complex64, as used by the mixed-precision path
 * (Section 6's per-mode LU at reduced precision, refined in FP64 by the
 * solve): the trailing-submatrix updates run on the tensor cores with every
 * FP32 operand split exactly into three BF16 pieces and the six piece
 * products of FP32 weight accumulated in FP32, so the factors carry FP32-grade
 * backward error.  Layout and outputs as mueller_lu_batched.  Returns
 * MUELLER_ETIMEOUT if a bounded device-side wait of the update gave up (the
 * factors are then unusable).  Synchronises `stream`. */
int mueller_lu_batched_c64(mueller_c64* A_dev, int n, int batch, int* piv_dev, int* info_dev, void* stream);

/* Device bytes of mueller_build for a body of N nodes and modes 0..M at the
 * given precision option: the return value is the peak during the build
 * (matrices, complex64 factors, residual slices and the near-panel spectra
 * scratch), *resident (if not null) what the context holds afterwards.  Used
 * to admit bodies under a memory budget; 0 for invalid sizes. */
size_t mueller_build_bytes(int N, int M, int precision, size_t* resident);

/* Peak device bytes of mueller_build_many for bodies of N[i] nodes and modes
 * 0..M[i]: what every body holds through the wave's factorization (its
 * resident bytes and LU workspace) plus the largest assembly-time surplus of
 * one body (bodies are assembled one after another).  0 for invalid sizes. */
size_t mueller_build_many_bytes(int count, const int* N, const int* M, int precision);

/* The LU tile autotuner's decisions so far in this process: up to cap
 * entries, each the upper end of a trailing-size bucket (rest_hi) and of a
 * matrix-count bucket (count_hi), the column tile chosen (tile) and the
 * measured milliseconds per matrix of one split + update step with tiles 32,
 * 64 and 128 (ms_per_matrix[3k .. 3k+2]).  Returns the number of entries
 * written, -1 for invalid arguments. */
int mueller_lu_tile_table(int* rest_hi, int* count_hi, int* tile, float* ms_per_matrix, int cap);

/* Bytes of complex128 factors for one body: 16 (4N)^2 (2M+1), the admission
 * unit named by the serving workload (the GPU path stores M+1 of them). */
size_t mueller_footprint_bytes(int N, int M);

/* Device-memory cache.  Buffers of at least 64 MiB that a build, a solve or
 * a destroyed context releases are kept by the library (per device, up to
 * the cap) and reused for requests of the same size rounded up to 2 MiB, so
 * repeated builds of similar bodies skip the driver's allocation and
 * release of several GB each.  A release synchronizes the device first (as
 * cudaFree does).  When an allocation fails, the cache is emptied and the
 * allocation retried.  mueller_cache_limit sets the cap (default 32 GiB; 0
 * disables caching) and returns the previous one; mueller_cache_trim returns
 * every cached block to the driver; mueller_cache_bytes reports the bytes
 * held.  Callers that budget device memory themselves should leave the cap
 * as headroom or trim first. */
void mueller_cache_trim(void);
size_t mueller_cache_limit(size_t bytes);
size_t mueller_cache_bytes(void);

/* Measured FP64 arithmetic peak of the current device in TFLOP/s: the best
 * of five timed launches of a register loop of independent fused
 * multiply-adds (8 chains per thread, 8 CTAs of 256 threads per SM; 2 flops
 * per FMA).  The paper's kernel evaluation and assembly (Sections 4-5) run on
 * the FP64 pipe; this is the denominator of their roofline.  Runs on `stream`
 * and synchronises it (about 2 s). */
int mueller_fp64_peak(double* tflops, void* stream);

/* Condition estimate of every mode's system (the paper reports LAPACK
 * ZGESVX condition numbers of its mode-0 systems, Section 6): kappa[m] for
 * m = 0..M (host array, may be NULL) = ||A'_m||_inf times Hager's estimate
 * (the iteration of LAPACK's xLACN2) of ||A'_m^{-1}||_inf, from the build's
 * LU factors (complex64 ones on the mixed paths), A'_m the L2-weighted
 * matrix (mode -m has the same value: A'_{-m} is A'_m with rows and columns
 * multiplied by +-1).  The estimate is a lower bound, in practice within a
 * small factor.  Also sets kappa_mode0, kappa_max, kappa_max_mode and
 * ms_cond in the stats.  One CTA per mode; synchronises `stream`. */
int mueller_cond_estimate(mueller_ctx* ctx, double* kappa, void* stream);

/* Host-spilled factor cache.  mueller_ctx_spill copies every device buffer
 * of the context (factors, residual slices, geometry, pivots) to pinned host
 * memory on `stream`, waits for the copies and releases the device buffers,
 * so that a caller keeping many bodies (a serving cache) can park the factors
 * of a body it evicts in host memory, over the CPU-GPU link, instead of
 * destroying them; mueller_ctx_restore allocates device buffers again and
 * copies the factors back (bit-identical), far cheaper than a new build.
 * While spilled, mueller_solve, mueller_rhs_*, mueller_eval and
 * mueller_far_field* return MUELLER_EINVAL; stats report spilled = 1, the
 * host bytes, and device_bytes = 0.  Both calls synchronise `stream`; both
 * are no-ops when the context is already in the requested place.  ENOMEM
 * leaves the context where it was. */
int mueller_ctx_spill(mueller_ctx* ctx, void* stream);
int mueller_ctx_restore(mueller_ctx* ctx, void* stream);

/* Checkpoints.  mueller_ctx_save writes to `path` the build's inputs (curve,
 * media, M, options) and every device buffer of the context (from host memory
 * when spilled); mueller_ctx_load reads such a file, checks the inputs as
 * mueller_build does and allocates and fills the device buffers, giving a
 * context whose solves are bit-identical to the saved one's, without the
 * assembly and factorization.  The file format is this library's own (not
 * portable across versions of it); MUELLER_EINVAL on a file that does not
 * match, MUELLER_ENOMEM when the device cannot hold the factors. */
int mueller_ctx_save(const mueller_ctx* ctx, const char* path);
int mueller_ctx_load(const char* path, void* stream, mueller_ctx** out);

int mueller_stats_get(const mueller_ctx* ctx, mueller_stats* out);
void mueller_destroy(mueller_ctx* ctx);
const char* mueller_strerror(int status);
/* Message of the last failing call on this thread (empty if none). */
const char* mueller_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
