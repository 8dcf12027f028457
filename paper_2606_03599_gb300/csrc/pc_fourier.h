// Block Fourier transform, reference-medium preconditioner and symbol tables.
#pragma once

#include <cufft.h>

#include <vector>

#include "pc_internal.h"

namespace pc {

struct SymbolParams {
    int X, Y, Z;
    double q;         // 1 / (4 h_s) = N / 4
    double Ainv[9];   // (A_hat^-1)_{s m}
    double Cref[36];  // reference stiffness (hat units)
    double null_tol;  // |eta| below this marks a zero-derivative mode
};

struct FftPlan {
    int dtype;
    int nsys;
    cufftHandle h;
};

}  // namespace pc

struct Precond {
    ~Precond();
    // Per Bloch-vector slot (pc_grid::ks): phase tables, reference symbols and null modes, slot-major
    // with the strides tab_len, 9 n_b and 65; the pointers below address slot 0.
    int nslots = 0;
    int tab_len = 0;
    double2* d_tabs = nullptr;  // phase tables (device)
    const double2 *ea = nullptr, *eb = nullptr, *egh = nullptr, *egf = nullptr;
    const double2 *twa = nullptr, *twb = nullptr, *twk = nullptr;
    float2* d_tabs32 = nullptr;  // the same tables rounded to complex64 (complex64 transforms)
    const float2 *ea32 = nullptr, *eb32 = nullptr, *egh32 = nullptr;
    const float2 *twa32 = nullptr, *twb32 = nullptr, *twk32 = nullptr;
    double* d_Aref = nullptr;  // 9 reals per mode (Hermitian 3x3 reference symbol)
    float* d_Aref32 = nullptr; // the same table rounded to FP32 (complex64 preconditioning)
    int* d_null = nullptr;     // per slot: [0] = count, [1..64] = modes with a vanishing symbol
    std::vector<int> null_modes;                 // slot 0
    std::vector<std::vector<int>> null_slot;     // every slot
    double rho_ref = 1.0;
    double Cref[36];
    std::vector<pc::FftPlan> plans;
    void* d_work = nullptr;
    size_t work_bytes = 0;
    // own quarter-grid DFT (pc_bloch_dft.cu): the n-th roots e^{-2 pi i j / n}, n = N/2, in both
    // precisions, and the block ids 0..3 as device ints
    double2* d_wn = nullptr;
    float2* d_wn32 = nullptr;
    const double2* wn = nullptr;
    const float2* wn32 = nullptr;
    int* d_blockids = nullptr;
    bool own_dft = false;  // the own kernels handle this grid's size
};

namespace pc {
int precond_create(pc_grid* g);
int precond_workspace(pc_grid* g, int dtype, int nsys, void** W);
// z_s = P r_s for nsys contiguous systems (stride 3 n_b); d_sys_block[s] = block of system s;
// d_skip: optional per-system skip flags (nonzero = leave z_s untouched).
// With d_part non-null, also writes per-CTA partial sums of Re<r_s, z_s> at d_part[s * npart + cta]
// (npart returned in *npart_out, equal to unpack_ctas(3 n_b)).
// fp32_inner (complex128 vectors only, d_part required): the transforms and the symbol solve run
// in complex64; r is rounded once on the way in and z widened on the way out.
// d_sys_k: optional Bloch slot of each system (device; null = slot 0); slots other than 0 need the
// own transform kernels (precond_multi_k).
int precond_apply(pc_grid* g, int dtype, int nsys, const void* r, void* z, const int* d_sys_block,
                  const int* d_skip, double sigma, cudaStream_t s, double* d_part = nullptr,
                  int* npart_out = nullptr, bool fp32_inner = false, const int* d_sys_k = nullptr);
// True when systems of several Bloch slots can share one preconditioner launch on this grid.
bool precond_multi_k(const pc_grid* g);
int unpack_ctas(int64_t vs);
// Partial sums per system of the preconditioner's fused Re<r, z> (the stride its callers allocate).
int precond_partials(const pc_grid* g);
// Own quarter-grid DFT kernels (pc_bloch_dft.cu): supported lengths n = N/2 (n = n1 n2, factors <= 16).
bool bloch_dft_supported(int n, int* n1, int* n2);
int bloch_dft_partials(int n);
// wdt: work precision, vdt: vector precision (PC_C64 / PC_C128); scale = 1 / n_b.
// sys_k: Bloch slot of each system (device, may be null = slot 0).
int own_precond(int n, int wdt, int vdt, int nsys, const void* r, void* z, void* W, const Precond* P,
                const int* sys_block, const int* sys_k, const int* skip, double shift_rho, double scale,
                double* part, cudaStream_t s);
int own_block_fourier(int n, int dtype, int inverse, const void* in, void* out, void* W, const Precond* P,
                      const int* d_block, int kslot, double scale, cudaStream_t s);
// kslot: the Bloch slot whose tables are used (slot 0 for the grid's current vector).
int block_fourier(pc_grid* g, int block, int dtype, int inverse, const void* in, void* out, cudaStream_t s,
                  int kslot = 0);
}  // namespace pc
