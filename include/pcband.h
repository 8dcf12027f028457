/*
 * pcband.h -- C ABI of the GB300 parity-blocked band solver.
 *
 * The library computes, for a Bloch vector kappa, the discrete elastic pencil
 *     A_h(kappa) v = omega^2 M_h v,   A_h = B_h C_h B_h^H
 * of the rotated staggered discretisation (Sec. 3, Eq. discrete_GEP) restricted
 * to one of the four parity blocks of even grids (Sec. 4, Theorem 4.1,
 * Cor. 4.2), and drives it with a shift-invert Krylov-Schur eigensolver whose
 * inner linear solves are preconditioned CG (Sec. 6, Eq.
 * shift_invert_system_unified).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid:      N x N x N nodes, N even and >= 4; node (i, j, k) sits at reduced
 *            coordinate (i, j, k)/N; full-grid order l = i + N (j + N k)
 *            (Eq. H_def: i fastest).
 * Blocks:    block b = 2 p12 + p13 holds the nodes with (i+j) mod 2 = p12 and
 *            (i+k) mod 2 = p13, i.e. the common eigenspace of Gamma_12,
 *            Gamma_13 with signs ((-1)^p12, (-1)^p13) (Eqs. V_sigma_main,
 *            Proj_sigma_main).  b = 0,1,2,3 <-> V_{++}, V_{+-}, V_{-+}, V_{--}.
 *            Block b has n_b = N^3/4 nodes; its canonical order t lists them by
 *            ascending full index l, which is t = i' + (N/2)(j'' + (N/2) k) with
 *            i = 2 i' + ((k + p13) mod 2), j = 2 j'' + ((k + p12 + p13) mod 2).
 *            block = -1 selects the full space (all n = N^3 nodes, order l).
 * Vectors:   complex, component-major: x[alpha * m + t], alpha = 0,1,2 the
 *            Cartesian velocity component, m = n_b (block) or n (full space).
 *            PC_C64 = interleaved float (re, im); PC_C128 = interleaved double.
 *            Vector arguments are DEVICE pointers owned by the caller; the
 *            library never frees them.
 * Units:     the library non-dimensionalises (Sec. 7.1, "after
 *            nondimensionalization"): stiffness C/C0 with C0 = 1e9 Pa, density
 *            rho/rho0 with rho0 = 1e3 kg/m^3, lengths /L with
 *            L = |det A_lat|^(1/3).  Operators applied through this ABI are
 *            A_hat = A_h L^2 / C0 and M_hat = M_h / rho0; eigenvalues of the
 *            hat pencil relate to SI as lambda_SI = lambda_hat C0 / (rho0 L^2).
 *            pc_eigs returns SI values (rad^2/s^2).
 * Streams:   `stream` is a cudaStream_t (0 = legacy default stream).  Calls
 *            that take a stream only enqueue work on it; they do not
 *            synchronise unless stated.
 * Errors:    every function returns PC_OK (0) or a negative PC_E* code; the
 *            message of the last failure on the calling thread is returned by
 *            pc_last_error().  No call aborts the process or traps the GPU:
 *            device loops carry iteration caps and report through status codes.
 * Threads:   a pc_grid handle must not be used by two threads at once; any
 *            number of handles may coexist.
 * Environment (read once per process; results do not depend on them):
 *            PC_APPLY_KERNEL = legacy | tma | split | row forces one stencil-
 *            kernel family for A/B comparisons (default: the plane-pipelined
 *            kernel for complex64 parity blocks, the two-pass kernels for
 *            complex128, or the autotuner's choice); PC_PCG_GRAPHS = 0 turns off CUDA-graph replay of PCG
 *            iterations; PC_TUNE_CACHE names the autotuner's cache file
 *            (pc_autotune); PC_WAIT_LIMIT = n sets how many polls a kernel's
 *            wait on its own shared-memory copies makes before it gives up
 *            (default 2^26; see pc_device_status).
 * Device waits: kernels that stage data through bulk or tensor copies wait
 *            on them with a bounded number of polls.  When a wait runs out the
 *            kernel lets its copies in flight land, records the event in the
 *            grid's device error word and returns, leaving its part of the
 *            output unwritten (inner products: NaN).  pc_shift_invert_pcg and
 *            pc_eigs read and clear that word before they return and then fail
 *            with PC_ECUDA; pc_device_status does the same for applies.
 */
#ifndef PCBAND_H
#define PCBAND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PC_OK 0
#define PC_EINVAL (-1)      /* bad argument: odd/small N, block, dtype, null pointer */
#define PC_ENOMEM (-2)      /* device or host allocation failed */
#define PC_ECUDA (-3)       /* a CUDA or cuFFT call failed */
#define PC_ENOCONV (-4)     /* iteration cap reached; outputs hold the best iterate */
#define PC_EBREAKDOWN (-5)  /* PCG found p^H (A - sigma M) p <= 0: shifted operator not SPD */
#define PC_ENAN (-6)        /* NaN or Inf met in a reduction */
#define PC_ESTATE (-7)      /* call out of order (e.g. apply before pc_set_k) */

/* ---- element types ----------------------------------------------------- */
#define PC_C64 1   /* complex64: FP32 storage and FP32 arithmetic */
#define PC_C128 2  /* complex128: FP64 storage and FP64 arithmetic */

/* ---- precision of pc_eigs ---------------------------------------------- */
#define PC_PREC_FP64 0   /* FP64 operator, inner PCG iterates, Krylov recurrences and residuals; the
                            Fourier preconditioner of the inner PCG runs in complex64 unless
                            pc_options.precond_fp32 = 0 (then every step is FP64) */
#define PC_PREC_MIXED 1  /* complex64 inner PCG, FP64 outer Krylov + residual refinement */

typedef struct pc_grid pc_grid; /* opaque, owned by the library */

/* Two-phase material, copied at pc_grid_create (caller keeps ownership). */
typedef struct {
    double rho[2];         /* density of phase 0 (matrix) and phase 1 (inclusion), kg/m^3 */
    double C[2][36];       /* 6x6 Voigt stiffness per phase, row-major, order [11,22,33,23,13,12],
                              engineering shear (Sec. 2, Eq. constitutive_voigt_main), Pa; symmetric */
    const uint8_t* phase;  /* host, N^3 phase ids (0/1) in full order, or NULL */
    const float* theta;    /* host, N^3 inclusion fractions in [0,1] (Eq. subpixel_material_average),
                              or NULL; at most one of phase/theta non-NULL; both NULL = phase 0 */
    double a_lat[9];       /* lattice basis A_lat = [a1 a2 a3], column-major: a_lat[3*l + r] = (a_l)_r, m */
} pc_material;

/* Outcome of one PCG solve. */
typedef struct {
    int iters;          /* iterations taken */
    int status;         /* PC_OK, PC_ENOCONV, PC_EBREAKDOWN or PC_ENAN */
    double rel_resid;   /* final ||r|| / ||rhs|| (recurrence residual) */
} pc_pcg_info;

/* Options of pc_eigs; fill with pc_options_default first. */
typedef struct {
    double tol;          /* converged when the true relative residual
                            ||A x - lambda M x|| / (max(|lambda|, |sigma|) ||M x||) <= tol (FP64),
                            i.e. relative to lambda wherever lambda >= |sigma| and to the shift's
                            scale for the acoustic modes next to Gamma; default 1e-8 */
    double inner_tol;    /* relative residual of each shift-invert solve; default 1e-10 */
    int precision;       /* PC_PREC_FP64 or PC_PREC_MIXED */
    int full_space;      /* 0: four parity blocks merged (default); 1: one full-space solve */
    int block_size;      /* Krylov block width per parity block; default 2 */
    int max_basis;       /* Krylov-Schur basis size before restart; default 24, raised where a
                            space's wanted pairs need more (their count + 2 blocks + 8) */
    int max_restarts;    /* outer iteration cap; default 60 */
    int inner_maxit;     /* PCG iteration cap per solve; default 400 */
    int guard;           /* extra Ritz pairs carried per block beyond its share; default 3 */
    int verbose;         /* 0 = silent */
    void* stream;        /* cudaStream_t for all of the solve's work, or NULL for an internal stream */
    int autotune;        /* 1 = time the stencil launch shapes for this grid's batches before solving
                            (pc_autotune); 0 = built-in choice.  Default 0 */
    int precond_fp32;    /* PC_PREC_FP64 only: 1 = the FP64 inner PCG applies its Fourier preconditioner
                            in complex64 (transforms, symbol solve) and uses the flexible CG beta; the
                            iterates, the stencil and the residuals stay FP64, so the solve reaches the
                            same inner_tol (the preconditioner only changes the iteration count).
                            0 = preconditioner in FP64.  Default 1 */
    int kbatch;          /* pc_eigs_batch only: Bloch vectors of one grid solved together in lockstep
                            (pc_eigs_multi) per work item; 0 = chosen per grid size (about 2^22 nodes
                            of systems per launch, at most 16), 1 = one at a time.  Default 0 */
} pc_options;

/* Statistics of one pc_eigs call. */
typedef struct {
    int status;              /* PC_OK or PC_ENOCONV */
    int outer_iters;         /* Krylov-Schur expansions, summed over blocks */
    int inner_solves;        /* shift-invert solves, summed over blocks */
    long long pcg_iters;     /* PCG iterations summed over all solves (and right-hand sides) */
    int max_pcg_iters;       /* longest single solve */
    int zero_modes;          /* zero-derivative modes deflated (12 full / 3 per block at Gamma) */
    double max_rel_resid;    /* largest true relative residual among returned pairs */
    double seconds;          /* wall time of the call */
} pc_eigs_info;

/* ---- lifecycle --------------------------------------------------------- */

/* Create a grid: copies the material to the device (phase ids or fractions in
 * full order and in the four block orders).  N even, >= 4.  *out receives the
 * handle.  Allocates device memory with cudaMalloc on the current device. */
int pc_grid_create(int N, const pc_material* m, pc_grid** out);

/* Create a grid with a nodewise material: every node l (full order) has its own stiffness and
 * density, the general pencil of Eq. discrete_GEP (C_h and M_h nodewise, Sec. 2-3) of which the
 * two-phase rule of pc_grid_create (Eq. subpixel_material_average) is the special case.
 * C21: host [N^3][21], the independent entries C_l[p][r], p <= r, of each node's symmetric 6x6
 * Voigt stiffness in row order ([11,22,33,23,13,12], engineering shear, Pa); rho: host [N^3],
 * kg/m^3, positive; a_lat as in pc_material.  Both arrays are copied (caller keeps ownership).
 * The device holds 22 FP64 values per node in each layout (about 0.35 KB per node in all).
 * Supported paths: complex128 applies (two-pass kernels), PC_PREC_FP64 eigen-solves, PCG,
 * mass, gradients (pc_eig_grad); complex64 applies and PC_PREC_MIXED return PC_EINVAL.  The
 * preconditioner's reference medium and the default shift use the nodes' volume averages and
 * largest entries.  PC_EINVAL for a non-finite entry or a non-positive density. */
int pc_grid_create_nodewise(int N, const double* C21, const double* rho, const double a_lat[9], pc_grid** out);

/* Release every device and host resource of the grid.  NULL is accepted. */
int pc_grid_destroy(pc_grid* g);

/* Scales of the non-dimensional units used by apply/PCG (see Units above). */
int pc_grid_units(const pc_grid* g, double* C0, double* rho0, double* L);

/* Set the Bloch vector: kappa in reduced reciprocal coordinates, phase
 * phi_l = 2 pi kappa_l across the l-th lattice translation (Eqs.
 * reduced_bloch_coordinate, phi_def).  Each kappa_l is first reduced into
 * [0, 1): the operator depends on exp(i phi_l) only, and the reduction fixes the
 * labelling of the Bloch Fourier modes alpha_p = (phi_1 + 2 pi p)/N etc. used by
 * pc_block_fourier.  Rebuilds the per-k Fourier symbol tables of the
 * preconditioner (Sec. 5.3, Eq. Bhat_xi_m_def). Synchronous. */
int pc_set_k(pc_grid* g, const double kappa[3]);

/* Host-only index map (no GPU needed): full_node_of_t[t] = full index l of
 * position t of block b, for t < N^3/4 (ascending l; Sec. 4, Eq. V_sigma_main).
 * full_node_of_t is caller-owned host memory of N^3/4 entries.  Takes the grid
 * size N rather than a grid handle: the map depends on N only, and taking N
 * lets it run without a device. */
int pc_block_index(int N, int block, int64_t* full_node_of_t);

/* ---- operator ---------------------------------------------------------- */

/* y = (A_hat - shift M_hat) x on block b (0..3) or the full space (b = -1):
 * the matrix-free chain x -> B^H x -> C B^H x -> B C B^H x of Sec. 6.1 with
 * Bloch-phased body-diagonal differences (Eqs. Sd_def, Dd_def,
 * Dtilde_recon_main, Dcal_cartesian_transform_main, B_discrete_main).
 * x, y: device, 3*m elements of `dtype`, must not overlap.  Enqueued on stream. */
int pc_block_apply(pc_grid* g, int block, int dtype, const void* x, void* y, double shift,
                   void* stream);

/* Same as pc_block_apply for `count` vectors of one block at once:
 * x and y hold `count` consecutive vectors of 3*m elements each. */
int pc_block_apply_many(pc_grid* g, int block, int dtype, int count, const void* x, void* y,
                        double shift, void* stream);

/* Status of the device work enqueued on `stream` for grid g: synchronises the
 * stream, then reads and clears the grid's device error word.  PC_OK, or
 * PC_ECUDA when a kernel's bounded wait on its own copies expired since the
 * last check (the outputs of the launches since then are incomplete). */
int pc_device_status(pc_grid* g, void* stream);

/* Apply M_hat (nodewise density, Eq. discrete_GEP) to a block vector. */
int pc_block_mass(pc_grid* g, int block, int dtype, const void* x, void* y, void* stream);

/* Gather block b of a full-space vector (Q_sigma^T x, Eq. Asigma_main) or
 * scatter a block vector into a full-space vector (Q_sigma y; other blocks'
 * entries untouched).  direction 0 = full->block, 1 = block->full. */
int pc_block_transfer(pc_grid* g, int block, int dtype, int direction, const void* src, void* dst,
                      void* stream);

/* Block Bloch Fourier transform (Sec. 5.2, Eq. Tsigma_unified): forward
 * (inverse = 0) computes what = T_sigma^H w, inverse computes w = T_sigma what.
 * Mode order (p fastest, then q, then r) with p, q < N/2, r < N.  dtype PC_C128
 * or PC_C64.  Requires pc_set_k. */
int pc_block_fourier(pc_grid* g, int block, int dtype, int inverse, const void* w, void* what,
                     void* stream);

/* Reference-medium preconditioner of the inner solves (Sec. 5.4), applied once:
 *   z = T_sigma diag_m (B_hat(m) C_ref B_hat(m)^H - sigma rho_ref I_3)^-1 T_sigma^H r
 * over the block's representative modes m (Eqs. Bhat_xi_m_def, Tsigma_unified), with C_ref
 * and rho_ref the volume averages of the stiffness and the density in hat units.  This is the
 * Psi-weighted Fourier SVD of Eq. weighted_svd_unified with Psi = C_ref^-1: the SVD
 * B_hat(m) C_ref^(1/2) = P Sigma Q^H gives B_hat C_ref B_hat^H = P Sigma^2 P^H, so each mode's
 * factor is P (Sigma^2 - sigma rho_ref)^-1 P^H.  For a homogeneous medium z solves
 * (A_hat - sigma M_hat) z = r exactly.
 * block: 0..3 (r, z block vectors [3][N^3/4]) or -1 (full-space vectors [3][N^3], handled as
 * its four blocks).  dtype PC_C64 or PC_C128.  fp32_transforms (PC_C128 only; ignored for
 * PC_C64): run the transforms and the 3x3 solves in complex64 on r rounded once and widen z,
 * as the FP64 solver does by default (pc_options.precond_fp32).  sigma: hat units, finite;
 * below the lowest eigenvalue keeps the factor positive definite.  r and z are caller-owned
 * device vectors and may be the same buffer.  Requires pc_set_k.  Stream-ordered; scratch
 * comes from the stream-ordered allocator and is released on the same stream. */
int pc_block_precond(pc_grid* g, int block, int dtype, int fp32_transforms, double sigma,
                     const void* r, void* z, void* stream);

/* ---- solvers ----------------------------------------------------------- */

/* Solve (A_hat - sigma M_hat) x = rhs on block b by PCG with the block Fourier
 * reference-medium preconditioner (Sec. 5.4, Sec. 6.1): x starts at zero and
 * stops at ||r|| <= tol ||rhs|| or maxit.  sigma must lie below the block's
 * lowest eigenvalue (the paper's sigma = -delta < 0); otherwise PCG may report
 * PC_EBREAKDOWN.  At Gamma the zero-derivative modes are not touched.
 * Synchronises the stream to fill `info` (may be NULL). */
int pc_shift_invert_pcg(pc_grid* g, int block, int dtype, double sigma, const void* rhs, void* x,
                        double tol, int maxit, pc_pcg_info* info, void* stream);

/* Fill `opt` with the defaults listed in pc_options. */
int pc_options_default(pc_options* opt);

/* Default shift sigma = -delta with delta = 0.30 C_max / rho_max in the hat
 * units (Eq. num_shift_delta_rule, with density normalised by its maximum). */
double pc_default_sigma(const pc_grid* g);

/* Lowest `nev` non-zero eigenvalues of (A_h(kappa), M_h) (Sec. 6): sets kappa,
 * solves the four parity blocks with shift-invert Krylov-Schur and merges
 * their spectra (Eq. block_gep_impl_unified), or solves the full space when
 * opt->full_space.  At kappa = 0 (mod 1) the zero-derivative modes found by
 * the Fourier SVD of the symbol blocks (Sec. 6.2, Eq. gamma_null_space_main)
 * are M-orthogonally projected out and not reported.  sigma: shift-invert
 * target in hat units (pass NaN for pc_default_sigma).
 * evals: host, nev doubles, ascending, SI (rad^2/s^2).
 * evecs: NULL or device [nev][3][N^3] complex128, full-space layout, M_h-normalised.
 * block_of: NULL or host int[nev], source block of each value (-1 for full space).
 * info: NULL or statistics.  Synchronous. */
int pc_eigs(pc_grid* g, const double kappa[3], int nev, double sigma, const pc_options* opt,
            double* evals, void* evecs, int* block_of, pc_eigs_info* info);

/* pc_eigs at nk Bloch vectors of one grid at once (1 <= nk <= 32; the block subproblems of all
 * of them are independent, Sec. 6.3): the grid holds one Bloch slot per vector, every
 * (vector, parity block) pair is one space of the same shift-invert Krylov-Schur iteration, and
 * each expansion runs one batched inner PCG, one set of Gram / update launches and one true-
 * residual apply over all unfinished spaces, so a launch serves several Bloch vectors (each
 * stencil item and preconditioner system carries its slot).  Results equal nk pc_eigs calls up to
 * rounding (same start vectors, same tests).  kappas: host [nk][3].  evals: host [nk][nev];
 * evecs: NULL or device [nk][nev][3][N^3] complex128, full-space layout, M_h-normalised (zero for a
 * Bloch vector that did not converge); block_of: NULL or host [nk][nev]; info: NULL or nk entries -- status, zero_modes and
 * max_rel_resid per vector; outer_iters, inner_solves, pcg_iters, max_pcg_iters and seconds are
 * totals of the whole call, repeated in every entry.  Afterwards the grid's current Bloch vector
 * (pc_set_k) is kappas[0:3].  nk > 1 needs a grid whose block transform runs in the library's own
 * kernels (pc_eigs_multi_max > 1), else PC_EINVAL.  Returns PC_ENOCONV when some vector did not
 * converge (its info status says which; the others are valid).  Synchronous. */
int pc_eigs_multi(pc_grid* g, int nk, const double* kappas, int nev, double sigma, const pc_options* opt,
                  double* evals, void* evecs, int* block_of, pc_eigs_info* info);

/* Largest nk pc_eigs_multi accepts for this grid (32, or 1 when the grid's quarter-grid length
 * N/2 has a prime factor above 16 or exceeds 96). */
int pc_eigs_multi_max(const pc_grid* g);

/* Batched apply: one launch computes y_i = (A_hat - shift_i M_hat) x_i for
 * count vectors that may belong to different parity blocks (blocks[i] in 0..3),
 * or count full-space vectors (every blocks[i] = -1).  x, y: host arrays of
 * `count` device pointers (3 n_b or 3 n elements each); shifts: host array. */
int pc_apply_batch(pc_grid* g, int dtype, int count, const int* blocks, const void* const* x,
                   void* const* y, const double* shifts, void* stream);

/* Bloch slots: set slots 0 .. nk - 1 (1 <= nk <= 32) of the grid to the reduced Bloch vectors
 * kappas[3 i .. 3 i + 2] (host); slot 0 becomes the current vector of pc_set_k, and the phases and
 * preconditioner tables of every slot are rebuilt.  pc_set_k is the nk = 1 case. */
int pc_set_k_multi(pc_grid* g, int nk, const double* kappas);

/* pc_apply_batch with item i at the Bloch vector of slot kslots[i] (host; NULL = all slot 0):
 * y_i = (A_hat(kappa_{kslots[i]}) - shift_i M_hat) x_i.  The two-pass complex128 kernels and the
 * plane-pipelined complex64 kernel serve all slots in one launch; other launch shapes run once
 * per run of equal slots. */
int pc_apply_batch_k(pc_grid* g, int dtype, int count, const int* blocks, const int* kslots,
                     const void* const* x, void* const* y, const double* shifts, void* stream);

/* Allocation-free apply with inner product: y = (A_hat - shift M_hat) x on
 * block b (0..3) or the full space (-1), and *dot = Re <x, y> (x^H y), written
 * to `dot`, one double of caller-owned DEVICE memory.  The paper has no
 * counterpart of this call; it exists for callers that must not let a library
 * allocate device memory -- an application whose GPU memory is already handed
 * out by its own pool, or a latency-critical loop that cannot afford the
 * implicit device synchronisation of cudaMalloc/cudaFree.  Its scratch (one
 * partial sum per CTA) lives in a fixed static device array of 2048 doubles
 * (16 KiB) that every device loading the library holds until the process
 * exits; no call allocates or frees.  Limits: at most 2^24 nodes per call
 * (N <= 406 for a block, N <= 256 for the full space), else PC_EINVAL with the
 * reason; within that limit every grid size is accepted (the call picks a
 * launch of at most 2048 CTAs).  x and y must not overlap.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls on a device share the array: calls whose kernels overlap on the GPU
 * race and may return a wrong *dot, so order them on one stream.  Each call
 * rewrites every slot it reads (a CTA whose bounded copy wait expired writes
 * NaN into its slot), so no state carries over between calls; an expired wait
 * during the call also makes *dot NaN.  Enqueued on `stream`. */
int pc_block_apply_dot_noalloc(pc_grid* g, int block, int dtype, const void* x, void* y, double shift,
                               double* dot, void* stream);

/* ---- batches of grids and Bloch vectors -------------------------------- */

/* A copy of grid `src` (same size, material, lattice and units; no Bloch vector set, no solver
 * state).  Device memory of its own; destroy with pc_grid_destroy. */
int pc_grid_clone(const pc_grid* src, pc_grid** out);

typedef struct {
    pc_grid* grid;          /* caller-owned; only read (workers solve on their own copies) */
    int nk;                 /* Bloch vectors of this grid */
    const double* kappas;   /* host [nk][3], reduced coordinates as in pc_set_k */
    int nev;                /* eigenvalues per Bloch vector */
    double sigma;           /* shift-invert target, NaN = pc_default_sigma of the grid */
    double* evals;          /* host [nk][nev] output (SI, as pc_eigs) */
    int* block_of;          /* host [nk][nev] output or NULL */
    int* status;            /* host [nk] output (pc_eigs status per Bloch vector) or NULL */
} pc_batch_job;

typedef struct {
    int workers;            /* host worker threads used */
    int kpoints;            /* Bloch vectors solved */
    int failed;             /* of which with a nonzero status */
    long long pcg_iters;    /* total inner PCG iterations */
    double max_rel_resid;   /* largest true relative residual over all reported pairs */
    double seconds;         /* wall time */
} pc_batch_info;

/* Band solves for many (grid, Bloch vector) pairs (the batching of the parity-block method's
 * independent subproblems, Sec. 6.3): the Bloch vectors of each grid are cut into chunks of
 * opt->kbatch (0 = sized per grid) and every chunk is solved as pc_eigs_multi does (all blocks
 * of all its vectors in lockstep), by `workers` host threads (1..16), each with its own CUDA
 * stream and its own copy of the grid it works on, taking chunks largest grid first.  With opt->autotune the
 * launch shapes of every grid size are tuned before the workers start.  opt->stream, if set,
 * is used for the tuning only.  Returns PC_OK, PC_ENOCONV when some Bloch vectors did not
 * converge (their status says which, the others are valid), or the first hard error. */
int pc_eigs_batch(pc_batch_job* jobs, int njobs, const pc_options* opt, int workers, pc_batch_info* info);

/* ---- launch tuning ----------------------------------------------------- */

/* Autotuner of the stencil apply (no counterpart in the paper: an implementation choice).
 * Times every applicable kernel and launch shape (row-tile kernel with several persistent CTA
 * counts, TMA tile kernel, register-staged kernel, two-pass kernels; several k-chunkings) on scratch vectors for
 * batches of `nitems` (rounded up to a power of two, 1..64) vectors of precision `dtype` in the
 * parity-block layout (layout 0), the full-space layout (1) or both (2), and keeps the fastest
 * for every later apply, PCG and eigen-solve on grids of the same size, material kind and lattice
 * in this process.  With the environment variable PC_TUNE_CACHE naming a file, results are read
 * from it and appended to it (one JSON-style line per key).  Synchronises `stream`; allocates and
 * frees scratch (2 x nitems vectors).  Needs pc_set_k first. */
int pc_autotune(pc_grid* g, int dtype, int layout, int nitems, void* stream);

/* The launch configuration the library will use for a batch of `nitems` vectors of `dtype` in
 * layout 0 (blocks) or 1 (full): kind 0 = register-staged, 1 = TMA tile, 2 = row tile, 3 = two-pass
 * (fluxes once per node, then gather; the default for complex128), 4 = plane-pipelined (producer
 * warp + consumer warps; the default for complex64 parity blocks); tile shape code; planes per CTA
 * (tz; row and plane-pipelined kernels: least planes per CTA); CTAs of the launch (two-pass: of
 * its gather). */
int pc_tuned_config(const pc_grid* g, int dtype, int layout, int nitems, int* kind, int* shape, int* tz, int* ctas);

/* ---- differentiation --------------------------------------------------- */

/* Eigenvalue gradients with respect to the nodewise material (Hellmann-Feynman
 * for the pencil of Eq. discrete_GEP_main): for eigenpairs (lambda_v, x_v) with
 * x_v^H M_hat x_v = 1 (as pc_eigs returns them), accumulates
 *   dC[q][l]  += sum_v w_v d lambda_v / d C_l[p][r]   (q over the 21 upper-
 *                triangular entries (p <= r) in row order of the Voigt matrix,
 *                Pa^-1 x rad^2/s^2; off-diagonal entries count both C[p][r] and C[r][p])
 *   drho[l]   += sum_v w_v d lambda_v / d rho_l       (per kg/m^3)
 * with d lambda/d C_l[p][r] = Re(conj(e_p) e_r)(2 if p != r) for the strain
 * e = B^H x at node l, and d lambda / d rho_l = -lambda sum_alpha |x_alpha(l)|^2.
 * X: nvec device complex128 vectors of block `block` (0..3) or of the full space
 * (-1), at the Bloch vector last set on g; lambdas (SI) and weights: host arrays.
 * dC: device FP64 [21][N^3], drho: device FP64 [N^3], full-grid node order; the
 * call adds to them.  For a degenerate cluster pass all of its vectors with one
 * common weight (the gradient of the cluster's sum is basis independent). */
int pc_eig_grad(pc_grid* g, int block, int nvec, const void* X, const double* lambdas, const double* weights,
                double* dC, double* drho, void* stream);

/* ---- diagnostics ------------------------------------------------------- */

/* Process-wide counters of the library's own kernel launches (cuFFT
 * kernels excluded) and, while timing is enabled, the device time of the
 * stencil-apply launches measured with CUDA events on their launch stream. */
typedef struct {
    long long launches;        /* every kernel launch of this library */
    long long apply_launches;  /* stencil-apply launches (both precisions) */
    long long apply_timed[2];  /* timed apply launches: [0] complex64, [1] complex128 */
    double apply_ms[2];        /* their summed device time, ms */
    double apply_nodes[2];     /* nodes of the items they processed; an item skipped at run
                                  time (a converged system of a batched solve) counts none */
    double apply_nodes_launched[2]; /* nodes of all items the timed launches carried, skipped
                                       ones included */
} pc_stats;

/* Enable (1) or disable (0) event timing of apply launches.  Timing adds two
 * event records per apply launch, and a one-CTA counting kernel after each
 * launch whose items carry run-time skip flags. */
int pc_stats_timing(int enable);

/* Reset all counters. */
int pc_stats_reset(void);

/* Read the counters; synchronises the device first. */
int pc_stats_get(pc_stats* out);


/* Message of the last failure on the calling thread ("" if none). */
const char* pc_last_error(void);

/* Library version string. */
const char* pc_version(void);

/* FP64 FMA throughput of the current device (no counterpart in the paper: the denominator of
 * the FP64 roofline of the complex128 kernels).  Runs a kernel of independent FP64 FMA chains
 * on every SM, growing its length until one launch takes about seconds/4, and returns the best
 * rate of the later launches: *tflops = 2 x FMA/s / 1e12, *fma_per_s (may be NULL) the FP64
 * FMA instruction rate summed over all threads.  Allocates and frees 8 bytes; synchronises
 * the device's legacy default stream.  seconds in (0, 60]. */
int pc_fp64_peak(double seconds, double* tflops, double* fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* PCBAND_H */
