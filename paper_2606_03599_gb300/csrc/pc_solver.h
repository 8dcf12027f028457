// Solver-side declarations: batched PCG and the shift-invert Krylov-Schur driver.
#pragma once

#include <vector>

#include "pc_fourier.h"
#include "pc_internal.h"

namespace pc {

// Per-system PCG scalars (device).
struct PcgScal {
    double rz;     // Re <r, z>
    double pq;     // Re <p, (A - sigma M) p>
    double alpha;  // rz / pq
    double beta;   // rz_new / rz
    double rr;     // ||r||^2
    double bb;     // ||b||^2
    double thr;    // tol^2 ||b||^2: converged once ||r||^2 <= thr (set per solve, outside the graphs)
    int done;      // 1 once converged or failed
    int status;    // PC_OK, PC_ENOCONV, PC_EBREAKDOWN, PC_ENAN
    int iters;     // iterations taken
    int pad;
};

struct PcgResult {
    int iters;
    int status;
    double rel_resid;
};

// Device workspace of one batched PCG configuration.
struct PcgWork {
    int dtype = 0, cap = 0;  // systems the buffers hold
    int64_t vs = 0;          // elements per system vector (3 m)
    void *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr;
    double* part = nullptr;  // partial sums, [3][cap][npart_max]
    int npart_max = 0;
    PcgScal* sc = nullptr;   // [cap]
    int* done = nullptr;     // [cap] mirror of sc.done for skip flags
    int* blocks = nullptr;   // [4 cap] block of each preconditioner subsystem
    int* kslots = nullptr;   // [4 cap] Bloch slot of each preconditioner subsystem
    PcgScal* h_sc = nullptr; // pinned host mirror
    // CUDA graph of one chunk of PCG iterations, valid for the key it was captured with
    cudaGraphExec_t gexec = nullptr;
    std::vector<double> gkey;
    long long glaunches = 0;       // library kernel launches inside the graph
    long long gapply = 0;          // of which stencil applies
    struct TimedSet* gtimed = nullptr;
    void drop_graph();
    void release();
};

// Solve (A - sigma M) x_s = b_s for nsys systems of the same grid, stacked contiguously
// (stride 3 m elements); blocks[s] in -1..3 (all full-space or all blocks).  x starts at
// zero.  Per-system results in res (host, nsys entries).  pre32 (complex128 only): apply the
// preconditioner in complex64 and use the flexible (Polak-Ribiere) beta, which keeps CG
// convergent under the preconditioner's rounding; the iterates stay complex128.  kslots (host,
// optional): the Bloch slot of each system (several Bloch vectors of the grid in one solve).
int pcg_solve(pc_grid* g, int dtype, int nsys, const int* blocks, double sigma, const void* B, void* X,
              double tol, int maxit, PcgResult* res, cudaStream_t s, bool pre32 = false,
              const int* kslots = nullptr);

// z = P_ref r once, outside a solve (block 0..3, or -1 for the full space through its four
// blocks); fp32_inner as pre32 above.
int precond_once(pc_grid* g, int block, int dtype, bool fp32_inner, double sigma, const void* r, void* z,
                 cudaStream_t s);

// Launch one batch of stencil applies on grid g (items share the layout kind).
int grid_apply(pc_grid* g, int dtype, bool full, const ApplyItem* items, int nitems, double* dot_partials,
               int dot_stride, cudaStream_t s, const ApplyConfig* cfg_in);
const void* grid_mat(const pc_grid* g, int block);
int launch_mass(int dtype, const void* x, void* y, const void* mat, int matkind, double rho0, double rho1,
                int64_t m, cudaStream_t s, int nvec);
int launch_transfer(int dtype, const void* src, void* dst, int N, int b, int dir, cudaStream_t s);

// Tall-skinny complex128 products of the outer loop (pc_blas.cu).  Columns are consecutive
// vectors of 3 m elements (component-major, m nodes).
// d_out (device, rows x cols, column-major) = A^H W B with W = the nodal mass (node densities
// rho0 + theta (rho1 - rho0) from mat, repeated over the components) when mat is non-null, else
// the identity.  d_part: scratch of part_cap doubles for the partial sums.
int ts_gram(const double2* A, int rows, const double2* B, int cols, int64_t m, const void* mat, int matkind,
            double rho0, double rho1, double2* d_out, double* d_part, size_t part_cap, cudaStream_t s);
// C (vs x cols) = beta C + alpha A h with A (vs x k) and h (device, k x cols, column-major);
// C must not overlap A; with beta == 0 C is only written.
int ts_update(const double2* A, int k, const double2* d_h, int cols, double2* C, int64_t vs, double alpha,
              double beta, cudaStream_t s);

// The same two products for several spaces in one launch (jobs of equal vector length; the
// Gram jobs all weighted by their mat or all unweighted).  Results of a Gram job go to its out
// (device, rows x cols column-major).  An update job's C must not overlap its A.
struct GramJob {
    const double2* A;
    int rows;
    const double2* B;
    int cols;
    const void* mat;
    double2* out;
};
struct UpdateJob {
    const double2* A;
    int k;
    const double2* h;
    int cols;
    double2* C;
    double alpha, beta;
};
int ts_gram_batch(const GramJob* jobs, int njobs, int64_t m, int matkind, double rho0, double rho1, double* d_part,
                  size_t part_cap, cudaStream_t s);
int ts_update_batch(const UpdateJob* jobs, int njobs, int64_t vs, cudaStream_t s);

}  // namespace pc

struct Solver {
    pc::PcgWork pcg[2];  // complex64 / complex128 workspaces
    ~Solver();
};
