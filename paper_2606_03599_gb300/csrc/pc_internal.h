// Internal declarations of the pcband library (host side).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcband.h"

namespace pc {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define PC_CUDA_TRY(expr)                                      \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return ::pc::cuda_fail(_e, #expr); \
    } while (0)

#define PC_TRY(expr)                \
    do {                            \
        int _rc = (expr);           \
        if (_rc != PC_OK) return _rc; \
    } while (0)

// ---------------------------------------------------------------- device parameters
// Everything a stencil launch needs about one grid at one Bloch vector, passed
// by value (kernel parameter space).  R = float (complex64 path) or double.
template <typename R>
struct StencilParams {
    R C[2][36];   // stiffness per phase in hat units, times (N/4)^2 when the lattice is cubic
    R rho[2];     // density per phase in hat units
    R Mmix[9];    // Mmix[s*3+m] = (A_hat^-1)_{s m} / (4 h_s); unused when cubic
    R ph[3][2];   // (cos phi_l, sin phi_l)
    int ortho[2]; // 1 if phase p's C couples no normal strain to a shear stress and no two shears
                  // (orthotropic in the lattice axes: isotropic, cubic, ...): 12 of 36 entries non-zero
    int N;        // grid size
    int X, Y, Z;  // lattice extents of the vector layout (N/2, N/2, N) or (N, N, N)
};

// One vector to process in a batched stencil launch.
struct ApplyItem {
    const void* x;
    void* y;
    const void* mat;  // material of this layout (uint8 phase ids or float theta)
    double shift;     // y = (A - shift M) x
    int block;        // 0..3 or -1 (full)
    int dot_slot;     // >= 0: write <x, y> partials to dot scratch slot, else -1
    const int* skip;  // optional device flag: nonzero = skip this item (converged system)
    int kslot = 0;    // Bloch-vector slot of the grid (0 = the vector pc_set_k sets)
};

// Bloch-vector slots of one grid: a solve over several Bloch vectors at once keeps each vector's
// phases and preconditioner tables in its own slot, and items of one launch may differ in slot.
constexpr int kMaxKSlots = 32;

// ---------------------------------------------------------------- kernels (launch wrappers)
// Fused stencil apply over a batch of items sharing params and layout kind.
// shape: tile code (0 = 32x8, 1 = 16x8, 2 = 8x8, 3 = 4x4); tz: k-planes per CTA.
// dp: per-CTA partial sums of Re<x, y> (slot-major, stride ds) or nullptr.
int launch_apply_f32(bool full, bool cubic, int matkind, int shape, const StencilParams<float>& P,
                     const ApplyItem* items, int nitems, int tz, double* dp, int ds, cudaStream_t s);
int launch_apply_f64(bool full, bool cubic, int matkind, int shape, const StencilParams<double>& P,
                     const ApplyItem* items, int nitems, int tz, double* dp, int ds, cudaStream_t s);
int launch_apply_tma_f32(bool full, bool cubic, int matkind, int shape, const StencilParams<float>& P,
                         const ApplyItem* items, int nitems, int tz, double* dp, int ds, int* err, cudaStream_t s);
// Row-tile kernel (complex64 parity blocks): mats = row-padded material per item; ctas = persistent CTAs.
int launch_apply_row_f32(bool cubic, int matkind, const StencilParams<float>& P, const ApplyItem* items,
                         const void* const* mats, int nitems, int ctas, double* dp, int ds, int* err, cudaStream_t s);
int row_apply_ctas(int X, int Y, int Z, int matkind, int nitems, int minseg = 12);
// Plane-pipelined kernel (complex64 parity blocks, even X): producer warp + consumer warps.
// item_ph: (cos, sin) of the three Bloch phases of each item ([nitems][3][2]).
int launch_apply_pipe_f32(bool cubic, int matkind, const StencilParams<float>& P, const ApplyItem* items,
                          const double* item_ph, const void* const* mats, int nitems, int ctas, double* dp, int ds,
                          int* err, cudaStream_t s);
int pipe_apply_ctas(int X, int Y, int Z, int matkind, int nitems, int minseg = 12);
bool pipe_geom_ok(int X, int Y, int Z, int matkind);
bool row_geom_fits(int X, int Y, int Z, int matkind);
int device_sm_count();
int launch_apply_tma_f64(bool full, bool cubic, int matkind, int shape, const StencilParams<double>& P,
                         const ApplyItem* items, int nitems, int tz, double* dp, int ds, int* err, cudaStream_t s);
// Two-pass complex128 apply (fluxes once per node through memory): scratch of split_scratch_bytes.
// item_ph as for the plane-pipelined kernel (every item its own Bloch phases).
int launch_apply_split_f64(bool full, bool cubic, int matkind, const StencilParams<double>& P, const ApplyItem* items,
                           const double* item_ph, int nitems, void* scratch, size_t scratch_bytes, double* dp, int ds,
                           cudaStream_t s);
int launch_apply_split_f32(bool full, bool cubic, int matkind, const StencilParams<float>& P, const ApplyItem* items,
                           const double* item_ph, int nitems, void* scratch, size_t scratch_bytes, double* dp, int ds,
                           cudaStream_t s);
size_t split_scratch_bytes(int X, int Y, int Z, int nitems, int dtype);
int split_apply_ctas(int64_t m);

struct ApplyConfig {
    int shape = 0;     // tile code (of the TMA kernel when tma, else of the register-staged kernel)
    int tz = 1;        // planes per CTA
    int ctas = 1;      // CTAs per item (row kernel: CTAs of the persistent launch)
    bool tma = false;  // TMA-staged kernel (quarter grids of even width >= 8)
    bool row = false;  // row-tile kernel (complex64 parity blocks, X even)
    bool split = false;  // two-pass complex128 kernels (flux, then gather)
    bool pipe = false;   // plane-pipelined kernel (complex64 parity blocks, even X)
};
// Kind code of a configuration as pc_tuned_config reports it.
inline int config_kind(const ApplyConfig& c) {
    return c.pipe ? 4 : (c.split ? 3 : (c.row ? 2 : (c.tma ? 1 : 0)));
}
// scratch_ok = false: only kernels that need no scratch memory of their own (no two-pass apply).
ApplyConfig choose_apply_config(int X, int Y, int Z, int nitems, int dtype, bool blocks = false, int matkind = 0,
                                bool scratch_ok = true);
// Launch configuration for a grid layout: the autotuned one when present, else the heuristic.
ApplyConfig apply_config_for(const pc_grid* g, bool full, int nitems, int dtype);
bool tuned_config(int X, int Y, int Z, int dtype, bool full, int matkind, bool cubic, int nitems, ApplyConfig* out);
int autotune_layout(pc_grid* g, int dtype, bool full, int nitems, cudaStream_t s, int verbose);
int tile_tx(int shape);
int tile_ty(int shape);

// Stencil parameters from hat-unit material tables (Chat[2][36], rhohat[2]),
// (A_hat^-1)_{s m} row-major, grid size N and Bloch phases phi[3].  For a cubic
// lattice the factor (N/4)^2 of the two reconstructed derivatives is folded
// into C; otherwise Mmix = (A_hat^-1)_{s m} / (4 h_s) with h_s = 1/N.
template <typename R>
inline void make_stencil_params(StencilParams<R>& P, const double Chat[2][36], const double rhohat[2],
                                const double Ainv[9], bool cubic, int N, const double phi[3], int X,
                                int Y, int Z) {
    const double q = N / 4.0;
    for (int p = 0; p < 2; ++p)
        for (int e = 0; e < 36; ++e) P.C[p][e] = (R)(Chat[p][e] * (cubic ? q * q : 1.0));
    for (int p = 0; p < 2; ++p) P.rho[p] = (R)rhohat[p];
    for (int p = 0; p < 2; ++p) {
        bool o = true;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                const bool keep = (i < 3 && j < 3) || i == j;
                if (!keep && Chat[p][i * 6 + j] != 0.0) o = false;
            }
        P.ortho[p] = o ? 1 : 0;
    }
    for (int e = 0; e < 9; ++e) P.Mmix[e] = (R)(Ainv[e] * q);
    for (int l = 0; l < 3; ++l) {
        P.ph[l][0] = (R)std::cos(phi[l]);
        P.ph[l][1] = (R)std::sin(phi[l]);
    }
    P.N = N;
    P.X = X;
    P.Y = Y;
    P.Z = Z;
}

// Bounded device waits.  Every spin-wait of a kernel (an mbarrier poll on its own copies) gives
// up after wait_limit() polls, records 1 in the grid's device error word and returns; the copies
// it still has in flight are then awaited with kDrainLimit polls so that no copy lands in shared
// memory the CTA has released.  PC_WAIT_LIMIT (read once) overrides the default 2^26 polls.
constexpr uint32_t kDrainLimit = 1u << 26;
uint32_t wait_limit();
// Reads and clears the grid's device error word after the work queued on s (synchronises s):
// PC_OK, or PC_ECUDA with a message when a bounded device wait expired.
int grid_device_status(pc_grid* g, cudaStream_t s);

int voigt_upper_host(int p, int r);  // position of Voigt entry (p, r) among the 21 upper entries

// Density of node t in hat units for the three material kinds: 0 = phase ids (uint8), 1 =
// inclusion fractions (float), 2 = nodewise material (FP64, component-major [22][m], entry 21 the
// density).  m = nodes of the layout.
template <typename R>
__host__ __device__ inline R node_rho_hat(const void* mat, int matkind, R rho0, R rho1, int64_t m, int64_t t) {
    if (matkind == 2) return (R) static_cast<const double*>(mat)[21 * m + t];
    const R th = matkind ? (R) static_cast<const float*>(mat)[t] : (R) static_cast<const uint8_t*>(mat)[t];
    return rho0 + th * (rho1 - rho0);
}

// Launch accounting (pc_stats): every kernel launch of the library calls note_launch.
void note_launch(int n = 1);
void note_apply_launch(int n = 1);
bool timing_enabled();
void* timing_begin(cudaStream_t s);
// Ends a timed apply call of nitems items of nodes_per_item nodes each; items with a skip flag are
// counted on the device when they run.
void timing_end(void* h, cudaStream_t s, int kind, const ApplyItem* items, int nitems, double nodes_per_item);
// Timing of launches captured into a CUDA graph (read after each replay).
struct TimedSet;
TimedSet* timing_capture_begin();
void timing_capture_end(TimedSet* t);
void timing_replayed(TimedSet* t);
void timing_free(TimedSet* t);
long long launch_count();
long long apply_launch_count();

// Per-k rebuild of the preconditioner tables (every slot in use); release of solver workspaces.
int precond_set_k(pc_grid* g);
// Sets slots 0 .. nk - 1 to the reduced Bloch vectors kappas[3 i .. 3 i + 2] (slot 0 also becomes
// the grid's current vector) and rebuilds the per-slot tables.  nk in [1, kMaxKSlots].
int grid_set_kslots(pc_grid* g, int nk, const double* kappas);
// (cos, sin) of the three Bloch phases of a slot.
void slot_phases(const pc_grid* g, int slot, double ph[3][2]);
void release_solver_state(pc_grid* g);

// ---------------------------------------------------------------- grid object
struct GridK {  // per-Bloch-vector state
    bool set = false;
    uint64_t version = 0;  // incremented by every pc_set_k (captured graphs depend on it)
    double kappa[3] = {0, 0, 0};
    double phi[3] = {0, 0, 0};
    bool gamma = false;
};

}  // namespace pc

struct pc_grid {
    int N = 0, X = 0, Y = 0, Z = 0;
    int64_t n = 0, nb = 0;
    double C0 = 1e9, rho0 = 1e3, L = 1.0;
    double Chat[2][36];
    double rhohat[2];
    double Ainv[9];  // (A_hat^-1)_{s m}, row-major s*3+m
    bool cubic = true;
    int matkind = 0;  // 0 = uint8 phase ids, 1 = float theta, 2 = nodewise ([22][m] FP64)
    double sigma_cmax = 0.0, sigma_rmax = 0.0;  // largest |C| entry and density (hat units): default shift
    double mean_theta = 0.0;  // volume fraction of phase 1
    int* d_err = nullptr;     // device error word of the TMA kernels (timed-out waits)
    void* d_mat_full = nullptr;
    void* d_mat_blk[4] = {nullptr, nullptr, nullptr, nullptr};
    void* d_mat_row[4] = {nullptr, nullptr, nullptr, nullptr};  // block material, rows padded to 16 bytes
    int mat_pitch = 0;                                          // elements per padded row
    pc::GridK k;                    // the Bloch vector of slot 0 (pc_set_k)
    pc::GridK ks[pc::kMaxKSlots];   // all slots; ks[0] mirrors k
    int nk = 1;                     // slots in use
    uint64_t kset_version = 0;      // incremented whenever any slot changes
    pc::StencilParams<double> P64;
    pc::StencilParams<float> P32;
    // scratch owned by the grid
    pc::ApplyItem* d_items = nullptr;
    int items_cap = 0;
    double* d_dot = nullptr;
    int dot_cap = 0;
    void* d_split = nullptr;  // scratch of the two-pass complex128 apply (extended x and fluxes)
    size_t split_bytes = 0;
    // preconditioner / solver workspaces are attached by their modules
    struct Precond* pre = nullptr;
    struct Solver* sol = nullptr;
    int device = 0;
};
