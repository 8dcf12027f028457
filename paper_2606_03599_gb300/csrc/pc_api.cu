// C ABI: grid lifecycle, Bloch vector, index maps, operator entry points.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pc_internal.h"
#include "pc_solver.h"

namespace pc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PC_ENOMEM : PC_ECUDA;
}


int tile_tx(int shape) { return shape == 0 ? 32 : shape == 1 ? 16 : shape == 2 ? 8 : 4; }
int tile_ty(int shape) { return shape <= 2 ? 8 : 4; }

static int apply_kernel_mode() {
    // PC_APPLY_KERNEL=legacy selects the register-staged kernel everywhere, =tma the TMA tile
    // kernel in place of the plane-pipelined kernel, =split the two-pass kernels for both
    // precisions, =row the row-tile kernel (A/B comparisons)
    static int mode = -1;
    if (mode < 0) {
        const char* v = std::getenv("PC_APPLY_KERNEL");
        const std::string m = v ? v : "";
        mode = m == "legacy" ? 1 : (m == "tma" ? 2 : (m == "split" ? 3 : (m == "row" ? 4 : 0)));
    }
    return mode;
}

uint32_t wait_limit() {
    static uint32_t lim = 0;
    static bool read = false;
    if (!read) {
        lim = 1u << 26;
        if (const char* v = std::getenv("PC_WAIT_LIMIT")) {
            char* end = nullptr;
            const unsigned long long n = std::strtoull(v, &end, 10);
            if (end != v && *end == 0 && n <= 0xffffffffull) lim = (uint32_t)n;
        }
        read = true;
    }
    return lim;
}

int grid_device_status(pc_grid* g, cudaStream_t s) {
    if (!g->d_err) return PC_OK;
    int h = 0;
    PC_CUDA_TRY(cudaMemcpyAsync(&h, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h == 0) return PC_OK;
    PC_CUDA_TRY(cudaMemsetAsync(g->d_err, 0, sizeof(int), s));
    PC_CUDA_TRY(cudaStreamSynchronize(s));
    return fail(PC_ECUDA, "a bounded device wait expired: the outputs of the launches since the last status "
                          "check are incomplete");
}

int device_sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                      cudaSuccess && v > 0)
            n = v;
        else
            n = 152;
    }
    return n;
}

ApplyConfig choose_apply_config(int X, int Y, int Z, int nitems, int dtype, bool blocks, int matkind, bool scratch_ok) {
    ApplyConfig c;
    if (scratch_ok && ((dtype == PC_C128 && (apply_kernel_mode() == 0 || matkind == 2)) || apply_kernel_mode() == 3)) {
        // complex128 is bound by GB300's FP64 pipe: fluxes once per node (two-pass kernels)
        c.split = true;
        c.shape = 0;
        c.tz = Z;
        c.ctas = split_apply_ctas((int64_t)X * Y * Z);
        return c;
    }
    if (apply_kernel_mode() == 0 && blocks && dtype == PC_C64 && pipe_geom_ok(X, Y, Z, matkind)) {
        // plane-pipelined kernel: persistent, whole rows per tile, producer warp + consumer warps
        c.pipe = true;
        c.shape = 0;
        c.tz = 12;  // planes per CTA at least
        c.ctas = pipe_apply_ctas(X, Y, Z, matkind, nitems, c.tz);
        return c;
    }
    if ((apply_kernel_mode() == 0 || apply_kernel_mode() == 4) && blocks && dtype == PC_C64 && X % 2 == 0 &&
        row_geom_fits(X, Y, Z, matkind)) {
        // row-tile kernel: persistent, whole rows per tile
        c.row = true;
        c.tma = false;
        c.shape = 0;
        c.tz = 12;  // planes per CTA at least
        c.ctas = row_apply_ctas(X, Y, Z, matkind, nitems, c.tz);
        return c;
    }
    if (apply_kernel_mode() != 1 && dtype == PC_C64 && X % 2 == 0 && X >= 8 && Y >= 8) {
        // TMA-staged kernel for complex64 (complex128 is FP64-ALU-bound on GB300 and runs faster on
        // the register-staged kernel): 16x16 tiles, else 8x8
        c.tma = true;
        // prefer a tile width that divides X (no idle columns); 16 when both do
        const int tx = (X % 16 == 0) ? 16 : (X % 8 == 0 ? 8 : (X >= 16 ? 16 : 8));
        c.shape = (tx == 16) ? 0 : 1;
        // tile height follows the shape code of launch_tma_shape: 16x16 / 16x8 or 8x8
        const int ty = (c.shape == 0 && dtype == PC_C64) ? 16 : 8;
        const int tiles = ((X + tx - 1) / tx) * ((Y + ty - 1) / ty);
        const long target = 2L * device_sm_count();  // two resident CTAs per SM: one full wave
        long nch = (target + (long)tiles * nitems - 1) / ((long)tiles * nitems);
        const long maxch = Z / 6 > 0 ? Z / 6 : 1;
        if (nch > maxch) nch = maxch;
        if (nch < 1) nch = 1;
        c.tz = (int)((Z + nch - 1) / nch);
        c.ctas = tiles * ((Z + c.tz - 1) / c.tz);
        return c;
    }
    c.tma = false;
    // widest tile whose a-extent divides X (no ragged tiles in a); FP64 capped at 16x8
    c.shape = 3;
    const int first = (dtype == PC_C128) ? 1 : 0;
    for (int s = first; s <= 2; ++s) {
        if (X % tile_tx(s) == 0 && X >= tile_tx(s) && Y >= tile_ty(s)) {
            c.shape = s;
            break;
        }
    }
    const int tiles = ((X + tile_tx(c.shape) - 1) / tile_tx(c.shape)) *
                      ((Y + tile_ty(c.shape) - 1) / tile_ty(c.shape));
    const long target = 4L * device_sm_count();  // about four resident CTAs per SM
    long nch = (target + (long)tiles * nitems - 1) / ((long)tiles * nitems);
    const long maxch = Z / 4 > 0 ? Z / 4 : 1;
    if (nch > maxch) nch = maxch;
    if (nch < 1) nch = 1;
    c.tz = (int)((Z + nch - 1) / nch);
    c.ctas = tiles * ((Z + c.tz - 1) / c.tz);
    return c;
}

int voigt_upper_host(int p, int r) {
    return p <= r ? p * 6 - p * (p - 1) / 2 + (r - p) : r * 6 - r * (r - 1) / 2 + (p - r);
}

static bool finite_all(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace pc

using namespace pc;

namespace pc {

// Bloch state of a reduced wave vector: phases of kappa mod 1, reduced first so that exact
// lattice vectors give phase 0.
static GridK make_gridk(const double kappa[3], uint64_t version) {
    GridK k;
    bool gamma = true;
    for (int l = 0; l < 3; ++l) {
        k.kappa[l] = kappa[l];
        const double frac = kappa[l] - std::floor(kappa[l]);
        k.phi[l] = 2.0 * M_PI * frac;
        if (frac != 0.0) gamma = false;
    }
    k.gamma = gamma;
    k.set = true;
    k.version = version;
    return k;
}

void slot_phases(const pc_grid* g, int slot, double ph[3][2]) {
    for (int l = 0; l < 3; ++l) {
        ph[l][0] = std::cos(g->ks[slot].phi[l]);
        ph[l][1] = std::sin(g->ks[slot].phi[l]);
    }
}

}  // namespace pc

static void fill_params(pc_grid* g) {
    make_stencil_params(g->P64, g->Chat, g->rhohat, g->Ainv, g->cubic, g->N, g->k.phi, g->X, g->Y, g->Z);
    make_stencil_params(g->P32, g->Chat, g->rhohat, g->Ainv, g->cubic, g->N, g->k.phi, g->X, g->Y, g->Z);
}

namespace pc {

int grid_set_kslots(pc_grid* g, int nk, const double* kappas) {
    if (!g || !kappas) return fail(PC_EINVAL, "set_k: null argument");
    if (nk < 1 || nk > kMaxKSlots) return fail(PC_EINVAL, "set_k: slot count out of range");
    if (!finite_all(kappas, 3 * nk)) return fail(PC_EINVAL, "set_k: non-finite kappa");
    const uint64_t v = g->k.version + 1;
    for (int i = 0; i < nk; ++i) g->ks[i] = make_gridk(kappas + 3 * i, v);
    g->k = g->ks[0];
    g->nk = nk;
    g->kset_version += 1;
    fill_params(g);
    return precond_set_k(g);
}

}  // namespace pc

extern "C" {

const char* pc_last_error(void) { return g_last_error.c_str(); }

const char* pc_version(void) { return "pcband 0.1 (sm_103a)"; }

int pc_block_index(int N, int block, int64_t* out) {
    if (N < 4 || (N & 1)) return fail(PC_EINVAL, "pc_block_index: N must be even and >= 4");
    if (block < 0 || block > 3) return fail(PC_EINVAL, "pc_block_index: block must be 0..3");
    if (!out) return fail(PC_EINVAL, "pc_block_index: null output");
    const int X = N / 2;
    const int p12 = block >> 1, p13 = block & 1;
    int64_t t = 0;
    for (int k = 0; k < N; ++k)
        for (int b = 0; b < X; ++b)
            for (int a = 0; a < X; ++a, ++t) {
                int64_t i = 2 * a + ((k + p13) & 1);
                int64_t j = 2 * b + ((k + p12 + p13) & 1);
                out[t] = i + (int64_t)N * (j + (int64_t)N * k);
            }
    return PC_OK;
}

int pc_grid_units(const pc_grid* g, double* C0, double* rho0, double* L) {
    if (!g) return fail(PC_EINVAL, "pc_grid_units: null grid");
    if (C0) *C0 = g->C0;
    if (rho0) *rho0 = g->rho0;
    if (L) *L = g->L;
    return PC_OK;
}

int pc_grid_destroy(pc_grid* g) {
    if (!g) return PC_OK;
    release_solver_state(g);
    cudaFree(g->d_mat_full);
    for (int b = 0; b < 4; ++b) cudaFree(g->d_mat_blk[b]);
    for (int b = 0; b < 4; ++b) cudaFree(g->d_mat_row[b]);
    cudaFree(g->d_dot);
    cudaFree(g->d_split);
    cudaFree(g->d_err);
    delete g;
    return PC_OK;
}

}  // extern "C"

// Lattice, grid size and units of a new grid (no material yet).  a_lat column-major.
static int grid_init(int N, const double a_lat[9], const char* who, pc_grid** gout) {
    *gout = nullptr;
    if (N < 4 || (N & 1)) return fail(PC_EINVAL, std::string(who) + ": N must be even and >= 4 (parity blocks need even grids)");
    if (N > 1024) return fail(PC_EINVAL, std::string(who) + ": N > 1024 not supported");
    if (!finite_all(a_lat, 9)) return fail(PC_EINVAL, std::string(who) + ": non-finite lattice basis");
    // A_lat (column-major input) and its determinant
    double A[3][3];
    for (int l = 0; l < 3; ++l)
        for (int r = 0; r < 3; ++r) A[r][l] = a_lat[3 * l + r];
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                 A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                 A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    if (!(std::fabs(det) > 0)) return fail(PC_EINVAL, std::string(who) + ": singular lattice basis");

    pc_grid* g = new pc_grid();
    g->N = N;
    g->X = N / 2;
    g->Y = N / 2;
    g->Z = N;
    g->n = (int64_t)N * N * N;
    g->nb = g->n / 4;
    g->L = std::cbrt(std::fabs(det));
    cudaGetDevice(&g->device);
    // inverse of A_hat = A_lat / L, row-major (A^-1)_{s m}
    double Ah[3][3];
    for (int r = 0; r < 3; ++r)
        for (int l = 0; l < 3; ++l) Ah[r][l] = A[r][l] / g->L;
    double dh = det / (g->L * g->L * g->L);
    double inv[3][3];
    inv[0][0] = (Ah[1][1] * Ah[2][2] - Ah[1][2] * Ah[2][1]) / dh;
    inv[0][1] = (Ah[0][2] * Ah[2][1] - Ah[0][1] * Ah[2][2]) / dh;
    inv[0][2] = (Ah[0][1] * Ah[1][2] - Ah[0][2] * Ah[1][1]) / dh;
    inv[1][0] = (Ah[1][2] * Ah[2][0] - Ah[1][0] * Ah[2][2]) / dh;
    inv[1][1] = (Ah[0][0] * Ah[2][2] - Ah[0][2] * Ah[2][0]) / dh;
    inv[1][2] = (Ah[0][2] * Ah[1][0] - Ah[0][0] * Ah[1][2]) / dh;
    inv[2][0] = (Ah[1][0] * Ah[2][1] - Ah[1][1] * Ah[2][0]) / dh;
    inv[2][1] = (Ah[0][1] * Ah[2][0] - Ah[0][0] * Ah[2][1]) / dh;
    inv[2][2] = (Ah[0][0] * Ah[1][1] - Ah[0][1] * Ah[1][0]) / dh;
    double dev = 0;
    for (int s = 0; s < 3; ++s)
        for (int mm = 0; mm < 3; ++mm) {
            g->Ainv[s * 3 + mm] = inv[s][mm];
            dev = std::fmax(dev, std::fabs(inv[s][mm] - (s == mm ? 1.0 : 0.0)));
        }
    g->cubic = dev < 1e-12;

    *gout = g;
    return PC_OK;
}

extern "C" {

int pc_grid_create(int N, const pc_material* m, pc_grid** out) {
    if (!out) return fail(PC_EINVAL, "pc_grid_create: null output");
    *out = nullptr;
    if (!m) return fail(PC_EINVAL, "pc_grid_create: null material");
    if (m->phase && m->theta) return fail(PC_EINVAL, "pc_grid_create: give phase or theta, not both");
    if (!finite_all(&m->C[0][0], 72) || !finite_all(m->rho, 2) || !finite_all(m->a_lat, 9))
        return fail(PC_EINVAL, "pc_grid_create: non-finite material constants");
    for (int p = 0; p < 2; ++p) {
        if (!(m->rho[p] > 0)) return fail(PC_EINVAL, "pc_grid_create: densities must be positive");
        double scale = 0;
        for (int e = 0; e < 36; ++e) scale = std::fmax(scale, std::fabs(m->C[p][e]));
        for (int a = 0; a < 6; ++a)
            for (int b = a + 1; b < 6; ++b)
                if (std::fabs(m->C[p][a * 6 + b] - m->C[p][b * 6 + a]) > 1e-12 * scale)
                    return fail(PC_EINVAL, "pc_grid_create: stiffness must be symmetric");
    }
    pc_grid* g = nullptr;
    PC_TRY(grid_init(N, m->a_lat, "pc_grid_create", &g));
    for (int p = 0; p < 2; ++p) {
        for (int e = 0; e < 36; ++e) g->Chat[p][e] = m->C[p][e] / g->C0;
        g->rhohat[p] = m->rho[p] / g->rho0;
    }
    for (int p = 0; p < 2; ++p) {
        for (int e = 0; e < 36; ++e) g->sigma_cmax = std::fmax(g->sigma_cmax, std::fabs(g->Chat[p][e]));
        g->sigma_rmax = std::fmax(g->sigma_rmax, g->rhohat[p]);
    }

    // material: full order and the four block orders
    g->matkind = m->theta ? 1 : 0;
    const size_t esz = g->matkind ? sizeof(float) : sizeof(uint8_t);
    std::vector<unsigned char> full(g->n * esz, 0);
    if (m->phase) {
        for (int64_t l = 0; l < g->n; ++l) {
            if (m->phase[l] > 1) {
                delete g;
                return fail(PC_EINVAL, "pc_grid_create: phase ids must be 0 or 1");
            }
            full[l] = m->phase[l];
        }
    } else if (m->theta) {
        for (int64_t l = 0; l < g->n; ++l)
            if (!(m->theta[l] >= 0.f && m->theta[l] <= 1.f)) {
                delete g;
                return fail(PC_EINVAL, "pc_grid_create: theta must lie in [0,1]");
            }
        std::memcpy(full.data(), m->theta, g->n * esz);
    }
    {
        double acc = 0.0;
        for (int64_t l = 0; l < g->n; ++l)
            acc += m->phase ? (double)m->phase[l] : (m->theta ? (double)m->theta[l] : 0.0);
        g->mean_theta = acc / (double)g->n;
    }
    cudaError_t e = cudaMalloc(&g->d_err, sizeof(int));
    if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(error word)"); }
    cudaMemset(g->d_err, 0, sizeof(int));
    e = cudaMalloc(&g->d_mat_full, g->n * esz);
    if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(material)"); }
    e = cudaMemcpy(g->d_mat_full, full.data(), g->n * esz, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMemcpy(material)"); }
    std::vector<int64_t> idx(g->nb);
    std::vector<unsigned char> blk(g->nb * esz);
    for (int b = 0; b < 4; ++b) {
        pc_block_index(N, b, idx.data());
        for (int64_t t = 0; t < g->nb; ++t) std::memcpy(&blk[t * esz], &full[idx[t] * esz], esz);
        e = cudaMalloc(&g->d_mat_blk[b], g->nb * esz);
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(block material)"); }
        e = cudaMemcpy(g->d_mat_blk[b], blk.data(), g->nb * esz, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMemcpy(block material)"); }
        // row-padded copy for the row-tile kernel: every quarter-grid row starts on a 16-byte boundary
        const int q = (int)(16 / esz);
        g->mat_pitch = (g->X + q - 1) / q * q;
        e = cudaMalloc(&g->d_mat_row[b], (size_t)g->mat_pitch * g->Y * g->Z * esz);
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(row material)"); }
        e = cudaMemset(g->d_mat_row[b], 0, (size_t)g->mat_pitch * g->Y * g->Z * esz);
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMemset(row material)"); }
        e = cudaMemcpy2D(g->d_mat_row[b], (size_t)g->mat_pitch * esz, blk.data(), (size_t)g->X * esz,
                         (size_t)g->X * esz, (size_t)g->Y * g->Z, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMemcpy2D(row material)"); }
    }
    fill_params(g);
    *out = g;
    return PC_OK;
}

int pc_grid_create_nodewise(int N, const double* C21, const double* rho, const double a_lat[9], pc_grid** out) {
    if (!out) return fail(PC_EINVAL, "pc_grid_create_nodewise: null output");
    *out = nullptr;
    if (!C21 || !rho || !a_lat) return fail(PC_EINVAL, "pc_grid_create_nodewise: null argument");
    pc_grid* g = nullptr;
    PC_TRY(grid_init(N, a_lat, "pc_grid_create_nodewise", &g));
    const int64_t n = g->n, nb = g->nb;
    // hat units; the reference medium (volume averages) doubles as both phase tables, which only the
    // preconditioner, the default shift and the launch parameters read for this material kind
    double Cavg[36] = {0}, ravg = 0.0;
    for (int64_t l = 0; l < n; ++l) {
        const double r = rho[l];
        bool ok = std::isfinite(r) && r > 0;
        for (int q = 0; q < 21; ++q) ok = ok && std::isfinite(C21[l * 21 + q]);
        if (!ok) {
            pc_grid_destroy(g);
            return fail(PC_EINVAL, "pc_grid_create_nodewise: non-finite stiffness or non-positive density at node " +
                                       std::to_string(l));
        }
        ravg += r / g->rho0;
        g->sigma_rmax = std::fmax(g->sigma_rmax, r / g->rho0);
        for (int p = 0; p < 6; ++p)
            for (int q = 0; q < 6; ++q) {
                const double c = C21[l * 21 + voigt_upper_host(p, q)] / g->C0;
                Cavg[p * 6 + q] += c;
                g->sigma_cmax = std::fmax(g->sigma_cmax, std::fabs(c));
            }
    }
    for (int p = 0; p < 2; ++p) {
        for (int e = 0; e < 36; ++e) g->Chat[p][e] = Cavg[e] / (double)n;
        g->rhohat[p] = ravg / (double)n;
    }
    g->mean_theta = 0.0;
    g->matkind = 2;
    // device layout [22][m]: the 21 entries scaled as the stencil tables (times (N/4)^2 on a cubic
    // lattice), then the density
    const double q2 = g->cubic ? (N / 4.0) * (N / 4.0) : 1.0;
    std::vector<double> full((size_t)22 * n);
    for (int64_t l = 0; l < n; ++l) {
        for (int q = 0; q < 21; ++q) full[(size_t)q * n + l] = C21[l * 21 + q] / g->C0 * q2;
        full[(size_t)21 * n + l] = rho[l] / g->rho0;
    }
    cudaError_t e = cudaMalloc(&g->d_err, sizeof(int));
    if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(error word)"); }
    cudaMemset(g->d_err, 0, sizeof(int));
    e = cudaMalloc(&g->d_mat_full, full.size() * sizeof(double));
    if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(material)"); }
    e = cudaMemcpy(g->d_mat_full, full.data(), full.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMemcpy(material)"); }
    std::vector<int64_t> idx(nb);
    std::vector<double> blk((size_t)22 * nb);
    for (int b = 0; b < 4; ++b) {
        pc_block_index(N, b, idx.data());
        for (int q = 0; q < 22; ++q)
            for (int64_t t = 0; t < nb; ++t) blk[(size_t)q * nb + t] = full[(size_t)q * n + idx[t]];
        e = cudaMalloc(&g->d_mat_blk[b], blk.size() * sizeof(double));
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMalloc(block material)"); }
        e = cudaMemcpy(g->d_mat_blk[b], blk.data(), blk.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { pc_grid_destroy(g); return cuda_fail(e, "cudaMemcpy(block material)"); }
    }
    fill_params(g);
    *out = g;
    return PC_OK;
}

int pc_set_k(pc_grid* g, const double kappa[3]) {
    if (!g || !kappa) return fail(PC_EINVAL, "pc_set_k: null argument");
    return grid_set_kslots(g, 1, kappa);
}

}  // extern "C"

namespace pc {

template <typename R>
static StencilParams<R> params_at(const pc_grid* g, const StencilParams<R>& base, int X, int Y, int Z, int slot) {
    StencilParams<R> P = base;
    P.X = X;
    P.Y = Y;
    P.Z = Z;
    double ph[3][2];
    slot_phases(g, slot, ph);
    for (int l = 0; l < 3; ++l) {
        P.ph[l][0] = (R)ph[l][0];
        P.ph[l][1] = (R)ph[l][1];
    }
    return P;
}

// One launch of items whose kernel takes grid-uniform Bloch phases (all items in `slot`), or, for
// the two-pass and plane-pipelined kernels, each item's own phases from item_ph.
static int apply_launch(pc_grid* g, int dtype, bool full, const ApplyConfig& cfg, const ApplyItem* items,
                        const double* item_ph, int nitems, int slot, double* dot_partials, int dot_stride,
                        cudaStream_t s) {
    const int X = full ? g->N : g->X, Y = full ? g->N : g->Y, Z = g->Z;
    if (cfg.split) {
        const size_t need = split_scratch_bytes(X, Y, Z, nitems, dtype);
        if (g->split_bytes < need) {
            // grown outside stream capture: the first launch of every batch shape runs eagerly
            cudaFree(g->d_split);
            g->d_split = nullptr;
            g->split_bytes = 0;
            cudaError_t e = cudaMalloc(&g->d_split, need);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(split apply scratch)");
            g->split_bytes = need;
        }
        if (dtype == PC_C64)
            return launch_apply_split_f32(full, g->cubic, g->matkind, params_at(g, g->P32, X, Y, Z, slot), items,
                                          item_ph, nitems, g->d_split, g->split_bytes, dot_partials, dot_stride, s);
        return launch_apply_split_f64(full, g->cubic, g->matkind, params_at(g, g->P64, X, Y, Z, slot), items,
                                      item_ph, nitems, g->d_split, g->split_bytes, dot_partials, dot_stride, s);
    }
    if (dtype == PC_C64 && (cfg.pipe || cfg.row)) {
        std::vector<const void*> mats(nitems);
        for (int i = 0; i < nitems; ++i) mats[i] = items[i].block >= 0 ? g->d_mat_row[items[i].block] : nullptr;
        const StencilParams<float> P = params_at(g, g->P32, X, Y, Z, slot);
        if (cfg.pipe)
            return launch_apply_pipe_f32(g->cubic, g->matkind, P, items, item_ph, mats.data(), nitems, cfg.ctas,
                                         dot_partials, dot_stride, g->d_err, s);
        return launch_apply_row_f32(g->cubic, g->matkind, P, items, mats.data(), nitems, cfg.ctas, dot_partials,
                                    dot_stride, g->d_err, s);
    }
    if (dtype == PC_C64) {
        const StencilParams<float> P = params_at(g, g->P32, X, Y, Z, slot);
        return cfg.tma ? launch_apply_tma_f32(full, g->cubic, g->matkind, cfg.shape, P, items, nitems, cfg.tz,
                                              dot_partials, dot_stride, g->d_err, s)
                       : launch_apply_f32(full, g->cubic, g->matkind, cfg.shape, P, items, nitems, cfg.tz,
                                          dot_partials, dot_stride, s);
    }
    const StencilParams<double> P = params_at(g, g->P64, X, Y, Z, slot);
    return cfg.tma ? launch_apply_tma_f64(full, g->cubic, g->matkind, cfg.shape, P, items, nitems, cfg.tz,
                                          dot_partials, dot_stride, g->d_err, s)
                   : launch_apply_f64(full, g->cubic, g->matkind, cfg.shape, P, items, nitems, cfg.tz, dot_partials,
                                      dot_stride, s);
}

// Launch one batch of stencil applies on grid g (items share the layout kind; each item at the
// Bloch vector of its slot).  The two-pass and plane-pipelined kernels take every item's phases,
// so one launch serves several Bloch vectors; the other kernels run once per run of equal slots.
int grid_apply(pc_grid* g, int dtype, bool full, const ApplyItem* items, int nitems, double* dot_partials,
               int dot_stride, cudaStream_t s, const ApplyConfig* cfg_in) {
    const int X = full ? g->N : g->X, Y = full ? g->N : g->Y, Z = g->Z;
    ApplyConfig cfg = cfg_in ? *cfg_in : apply_config_for(g, full, nitems, dtype);
    if (g->matkind == 2 && !(dtype == PC_C128 && cfg.split))
        return fail(PC_EINVAL, "apply: a nodewise material is applied by the complex128 two-pass kernels only");
    bool uniform = true;
    std::vector<double> iph((size_t)6 * std::max(nitems, 1));
    for (int i = 0; i < nitems; ++i) {
        const int ks = items[i].kslot;
        if (ks < 0 || ks >= g->nk) return fail(PC_EINVAL, "apply: item Bloch slot out of range");
        if (ks != items[0].kslot) uniform = false;
        slot_phases(g, ks, reinterpret_cast<double(*)[2]>(&iph[(size_t)6 * i]));
    }
    void* th = timing_enabled() ? timing_begin(s) : nullptr;
    int rc = PC_OK;
    const bool per_item = cfg.split || (dtype == PC_C64 && cfg.pipe);
    if (uniform || per_item) {
        rc = apply_launch(g, dtype, full, cfg, items, iph.data(), nitems, nitems ? items[0].kslot : 0, dot_partials,
                          dot_stride, s);
    } else {
        for (int i = 0; i < nitems && rc == PC_OK;) {
            int j = i;
            while (j < nitems && items[j].kslot == items[i].kslot) ++j;
            rc = apply_launch(g, dtype, full, cfg, items + i, iph.data() + 6 * i, j - i, items[i].kslot, dot_partials,
                              dot_stride, s);
            i = j;
        }
    }
    if (th) timing_end(th, s, dtype == PC_C64 ? 0 : 1, items, nitems, (double)X * Y * Z);
    return rc;
}

const void* grid_mat(const pc_grid* g, int block) { return block < 0 ? g->d_mat_full : g->d_mat_blk[block]; }

}  // namespace pc

extern "C" {

int pc_block_apply_many(pc_grid* g, int block, int dtype, int count, const void* x, void* y, double shift,
                        void* stream) {
    if (!g) return fail(PC_EINVAL, "pc_block_apply: null grid");
    if (block < -1 || block > 3) return fail(PC_EINVAL, "pc_block_apply: block must be -1..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_block_apply: dtype must be PC_C64 or PC_C128");
    if (!x || !y) return fail(PC_EINVAL, "pc_block_apply: null vector");
    if (count < 0) return fail(PC_EINVAL, "pc_block_apply: negative count");
    if (!std::isfinite(shift)) return fail(PC_EINVAL, "pc_block_apply: non-finite shift");
    if (!g->k.set) return fail(PC_ESTATE, "pc_block_apply: call pc_set_k first");
    if (count == 0) return PC_OK;
    const int64_t m = block < 0 ? g->n : g->nb;
    const size_t vbytes = 3 * m * (dtype == PC_C64 ? 8 : 16);
    const char* xb = static_cast<const char*>(x);
    char* yb = static_cast<char*>(y);
    if (xb < yb + vbytes * count && yb < xb + vbytes * count)
        return fail(PC_EINVAL, "pc_block_apply: x and y overlap");
    std::vector<ApplyItem> items(count);
    for (int i = 0; i < count; ++i) {
        items[i].x = xb + vbytes * i;
        items[i].y = yb + vbytes * i;
        items[i].mat = grid_mat(g, block);
        items[i].shift = shift;
        items[i].block = block;
        items[i].dot_slot = -1;
        items[i].skip = nullptr;
    }
    return grid_apply(g, dtype, block < 0, items.data(), count, nullptr, 0, (cudaStream_t)stream, nullptr);
}

int pc_apply_batch_k(pc_grid* g, int dtype, int count, const int* blocks, const int* kslots, const void* const* x,
                     void* const* y, const double* shifts, void* stream) {
    if (!g || !blocks || !x || !y || !shifts) return fail(PC_EINVAL, "pc_apply_batch: null argument");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_apply_batch: bad dtype");
    if (count < 0) return fail(PC_EINVAL, "pc_apply_batch: negative count");
    if (!g->k.set) return fail(PC_ESTATE, "pc_apply_batch: call pc_set_k first");
    if (count == 0) return PC_OK;
    const bool full = blocks[0] < 0;
    std::vector<ApplyItem> items(count);
    for (int i = 0; i < count; ++i) {
        if (blocks[i] < -1 || blocks[i] > 3 || (blocks[i] < 0) != full)
            return fail(PC_EINVAL, "pc_apply_batch: blocks must all be 0..3 or all -1");
        if (!x[i] || !y[i] || x[i] == y[i]) return fail(PC_EINVAL, "pc_apply_batch: null or aliased vector");
        if (!std::isfinite(shifts[i])) return fail(PC_EINVAL, "pc_apply_batch: non-finite shift");
        if (kslots && (kslots[i] < 0 || kslots[i] >= g->nk))
            return fail(PC_EINVAL, "pc_apply_batch: Bloch slot out of range");
        items[i].x = x[i];
        items[i].y = y[i];
        items[i].mat = grid_mat(g, blocks[i]);
        items[i].shift = shifts[i];
        items[i].block = blocks[i];
        items[i].dot_slot = -1;
        items[i].skip = nullptr;
        items[i].kslot = kslots ? kslots[i] : 0;
    }
    return grid_apply(g, dtype, full, items.data(), count, nullptr, 0, (cudaStream_t)stream, nullptr);
}

int pc_apply_batch(pc_grid* g, int dtype, int count, const int* blocks, const void* const* x, void* const* y,
                   const double* shifts, void* stream) {
    return pc_apply_batch_k(g, dtype, count, blocks, nullptr, x, y, shifts, stream);
}

int pc_set_k_multi(pc_grid* g, int nk, const double* kappas) {
    if (!g || !kappas) return fail(PC_EINVAL, "pc_set_k_multi: null argument");
    return grid_set_kslots(g, nk, kappas);
}

int pc_device_status(pc_grid* g, void* stream) {
    if (!g) return fail(PC_EINVAL, "pc_device_status: null grid");
    return grid_device_status(g, (cudaStream_t)stream);
}

int pc_block_apply(pc_grid* g, int block, int dtype, const void* x, void* y, double shift, void* stream) {
    return pc_block_apply_many(g, block, dtype, 1, x, y, shift, stream);
}

int pc_block_mass(pc_grid* g, int block, int dtype, const void* x, void* y, void* stream) {
    if (!g || !x || !y) return fail(PC_EINVAL, "pc_block_mass: null argument");
    if (block < -1 || block > 3) return fail(PC_EINVAL, "pc_block_mass: block must be -1..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_block_mass: bad dtype");
    const int64_t m = block < 0 ? g->n : g->nb;
    return launch_mass(dtype, x, y, grid_mat(g, block), g->matkind, g->rhohat[0], g->rhohat[1], m,
                       (cudaStream_t)stream, 1);
}

int pc_block_transfer(pc_grid* g, int block, int dtype, int direction, const void* src, void* dst,
                      void* stream) {
    if (!g || !src || !dst) return fail(PC_EINVAL, "pc_block_transfer: null argument");
    if (block < 0 || block > 3) return fail(PC_EINVAL, "pc_block_transfer: block must be 0..3");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_block_transfer: bad dtype");
    if (direction != 0 && direction != 1) return fail(PC_EINVAL, "pc_block_transfer: direction must be 0 or 1");
    return launch_transfer(dtype, src, dst, g->N, block, direction, (cudaStream_t)stream);
}

}  // extern "C"
