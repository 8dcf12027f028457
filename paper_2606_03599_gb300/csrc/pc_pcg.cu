// Batched preconditioned conjugate gradients for the shift-invert systems
// (A - sigma M) x = b of Sec. 6.1 (Eq. shift_invert_system_unified, with
// sigma = -delta), device-resident: every scalar of every system lives on the
// GPU, reductions are deterministic (fixed-order sums of per-CTA partials), and
// the host only polls the per-system done flags every few iterations.
//
// One iteration: q = (A - sigma M) p with fused partials of Re<p, q> (stencil
// kernel) -> alpha -> x += alpha p, r -= alpha q with partials of ||r||^2 ->
// z = P r (block Fourier preconditioner) with partials of Re<r, z> -> beta and
// the convergence test ||r|| <= tol ||b|| -> p = z + beta p.
#include <cstdlib>
#include <string>
#include <cmath>
#include <cstring>
#include <vector>

#include "pc_complex.cuh"
#include "pc_solver.h"

namespace pc {

__device__ __forceinline__ double block_sum_pcg(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// Fixed-order sum of n partials by one CTA (result in thread 0).
__device__ __forceinline__ double reduce_partials(const double* p, int n) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
    return block_sum_pcg(v);
}

template <typename C>
__global__ void pcg_start(const C* __restrict__ b, C* __restrict__ x, C* __restrict__ r, int64_t vs,
                          double* __restrict__ part, int npart) {
    const int s = blockIdx.y;
    using R = decltype(b[0].x);
    R acc = 0;  // per-thread sums in the working precision (complex64: FP32 accumulation), FP64 across threads
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        C v = b[s * vs + e];
        r[s * vs + e] = v;
        x[s * vs + e] = make_c<C>(0, 0);
        acc = cdotre(v, v, acc);
    }
    const double sum = block_sum_pcg((double)acc);
    if (threadIdx.x == 0) part[(int64_t)s * npart + blockIdx.x] = sum;
}

// bb = sum part_bb; init the scalars and flags: a zero right-hand side is solved by x = 0 and
// its system is retired before the first preconditioner application.  The convergence
// threshold tol2 bb is kept with the scalars, so that the captured iterations do not depend on
// the tolerance.
__global__ void pcg_start_bb(PcgScal* sc, int* done, const double* part_bb, int sbb, int nbb, double tol2) {
    const int s = blockIdx.x;
    double bb = reduce_partials(part_bb + (int64_t)s * sbb, nbb);
    if (threadIdx.x == 0) {
        PcgScal v;
        v.rz = 0;
        v.pq = 0;
        v.alpha = 0;
        v.beta = 0;
        v.rr = bb;
        v.bb = bb;
        v.thr = tol2 * bb;
        v.iters = 0;
        v.pad = 0;
        v.status = PC_OK;
        v.done = 0;
        if (!isfinite(bb)) {
            v.status = PC_ENAN;
            v.done = 1;
        } else if (bb == 0.0) {
            v.done = 1;  // zero right-hand side: x = 0 is exact
        }
        sc[s] = v;
        done[s] = v.done;
    }
}

// rz = sum part_rz of the systems still running.
__global__ void pcg_start_rz(PcgScal* sc, int* done, const double* part_rz, int nrz) {
    const int s = blockIdx.x;
    if (done[s]) return;
    double rz = reduce_partials(part_rz + (int64_t)s * nrz, nrz);
    if (threadIdx.x == 0) {
        PcgScal v = sc[s];
        v.rz = rz;
        if (!isfinite(rz)) {
            v.status = PC_ENAN;
            v.done = 1;
        } else if (!(rz > 0.0)) {
            v.status = PC_EBREAKDOWN;  // preconditioner not positive definite
            v.done = 1;
        }
        sc[s] = v;
        done[s] = v.done;
    }
}

template <typename C>
__global__ void pcg_copy(const C* __restrict__ z, C* __restrict__ p, int64_t vs, const int* __restrict__ done) {
    const int s = blockIdx.y;
    if (done[s]) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x)
        p[s * vs + e] = z[s * vs + e];
}

__global__ void pcg_alpha(PcgScal* sc, int* done, const double* part_pq, int spq, int npq) {
    const int s = blockIdx.x;
    if (done[s]) return;
    double pq = reduce_partials(part_pq + (int64_t)s * spq, npq);
    if (threadIdx.x == 0) {
        sc[s].pq = pq;
        if (!isfinite(pq)) {
            sc[s].status = PC_ENAN;
            sc[s].done = 1;
            done[s] = 1;
        } else if (!(pq > 0.0)) {
            sc[s].status = PC_EBREAKDOWN;
            sc[s].done = 1;
            done[s] = 1;
        } else {
            sc[s].alpha = sc[s].rz / pq;
        }
    }
}

// x += alpha p, r -= alpha q with partials of ||r||^2; with zold non-null also partials of
// Re<r_new, z_old> (flexible CG: the preconditioner is applied in lower precision).
template <typename C>
__global__ void pcg_update_xr(C* __restrict__ x, C* __restrict__ r, const C* __restrict__ p, const C* __restrict__ q,
                              const PcgScal* __restrict__ sc, const int* __restrict__ done, int64_t vs,
                              double* __restrict__ part, int npart, const C* __restrict__ zold,
                              double* __restrict__ part_d) {
    const int s = blockIdx.y;
    if (done[s]) return;
    using R = decltype(x[0].x);
    const R a = (R)sc[s].alpha;
    // per-thread sums in the working precision (complex64: FP32 accumulation), FP64 across threads
    R acc = 0, accd = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = s * vs + e;
        x[i] = cfma(a, p[i], x[i]);
        C rv = cfma(-a, q[i], r[i]);
        r[i] = rv;
        acc = cdotre(rv, rv, acc);
        if (zold != nullptr) accd = cdotre(rv, zold[i], accd);
    }
    const double sum = block_sum_pcg((double)acc);
    if (threadIdx.x == 0) part[(int64_t)s * npart + blockIdx.x] = sum;
    if (zold != nullptr) {
        const double sumd = block_sum_pcg((double)accd);
        if (threadIdx.x == 0) part_d[(int64_t)s * npart + blockIdx.x] = sumd;
    }
}

// beta = rz_new / rz_old (Fletcher-Reeves form), or with part_d non-null the flexible
// (Polak-Ribiere) form beta = (rz_new - Re<r_new, z_old>) / rz_old.
__global__ void pcg_beta(PcgScal* sc, int* done, const double* part_rr, int srr, int nrr, const double* part_rz,
                         int nrz, int maxit, const double* part_d) {
    const int s = blockIdx.x;
    if (done[s]) return;
    double rr = reduce_partials(part_rr + (int64_t)s * srr, nrr);
    double rz = reduce_partials(part_rz + (int64_t)s * nrz, nrz);
    double rzd = part_d != nullptr ? reduce_partials(part_d + (int64_t)s * srr, nrr) : 0.0;
    if (threadIdx.x == 0) {
        PcgScal v = sc[s];
        v.iters += 1;
        v.rr = rr;
        if (!isfinite(rr) || !isfinite(rz)) {
            v.status = PC_ENAN;
            v.done = 1;
        } else if (rr <= v.thr) {
            v.status = PC_OK;
            v.done = 1;
        } else if (v.iters >= maxit) {
            v.status = PC_ENOCONV;
            v.done = 1;
        } else if (!(rz > 0.0)) {
            v.status = PC_EBREAKDOWN;
            v.done = 1;
        } else {
            v.beta = (rz - rzd) / v.rz;
            v.rz = rz;
        }
        sc[s] = v;
        done[s] = v.done;
    }
}

template <typename C>
__global__ void pcg_update_p(C* __restrict__ p, const C* __restrict__ z, const PcgScal* __restrict__ sc,
                             const int* __restrict__ done, int64_t vs) {
    const int s = blockIdx.y;
    if (done[s]) return;
    using R = decltype(p[0].x);
    const R b = (R)sc[s].beta;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < vs; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = s * vs + e;
        p[i] = cfma(b, p[i], z[i]);
    }
}

// Gather/scatter between a full-space vector and its four block vectors (stacked).
template <typename C>
__global__ void full_to_blocks(const C* __restrict__ full, C* __restrict__ blk, int N, int nsys) {
    const int64_t n = (int64_t)N * N * N, nb = n / 4;
    const int X = N / 2;
    const int64_t total = (int64_t)nsys * 4 * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e % nb;
        const int b = (int)((e / nb) % 4);
        const int64_t s = e / (4 * nb);
        const int64_t a = t % X, bb = (t / X) % X, k = t / ((int64_t)X * X);
        const int p12 = b >> 1, p13 = b & 1;
        const int64_t l = (2 * a + ((k + p13) & 1)) + (int64_t)N * ((2 * bb + ((k + p12 + p13) & 1)) + (int64_t)N * k);
        for (int c = 0; c < 3; ++c) blk[(s * 4 + b) * 3 * nb + c * nb + t] = full[s * 3 * n + c * n + l];
    }
}

template <typename C>
__global__ void blocks_to_full(const C* __restrict__ blk, C* __restrict__ full, int N, int nsys) {
    const int64_t n = (int64_t)N * N * N, nb = n / 4;
    const int X = N / 2;
    const int64_t total = (int64_t)nsys * 4 * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e % nb;
        const int b = (int)((e / nb) % 4);
        const int64_t s = e / (4 * nb);
        const int64_t a = t % X, bb = (t / X) % X, k = t / ((int64_t)X * X);
        const int p12 = b >> 1, p13 = b & 1;
        const int64_t l = (2 * a + ((k + p13) & 1)) + (int64_t)N * ((2 * bb + ((k + p12 + p13) & 1)) + (int64_t)N * k);
        for (int c = 0; c < 3; ++c) full[s * 3 * n + c * n + l] = blk[(s * 4 + b) * 3 * nb + c * nb + t];
    }
}

// CUDA-graph replay of PCG iteration chunks (PC_PCG_GRAPHS=0 turns it off).
static bool pcg_graphs_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* v = std::getenv("PC_PCG_GRAPHS");
        on = (v && std::string(v) == "0") ? 0 : 1;
    }
    return on != 0;
}

static int vec_ctas(int64_t vs) {
    int64_t g = (vs + 1023) / 1024;
    if (g > 304) g = 304;
    return (int)(g < 1 ? 1 : g);
}

void PcgWork::drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    gkey.clear();
    glaunches = 0;
    gapply = 0;
    timing_free(gtimed);
    gtimed = nullptr;
}

void PcgWork::release() {
    drop_graph();
    cudaFree(R);
    cudaFree(Z);
    cudaFree(P);
    cudaFree(Q);
    cudaFree(part);
    cudaFree(sc);
    cudaFree(done);
    cudaFree(blocks);
    cudaFree(kslots);
    cudaFreeHost(h_sc);
    R = Z = P = Q = nullptr;
    part = nullptr;
    sc = nullptr;
    done = blocks = kslots = nullptr;
    h_sc = nullptr;
    cap = 0;
}

static int solver_get(pc_grid* g, Solver** out) {
    if (!g->sol) g->sol = new Solver();
    *out = g->sol;
    return PC_OK;
}

// Workspace for nsys systems of vs elements (+ block scratch for full-space preconditioning).
static int pcg_work(pc_grid* g, int dtype, int nsys, int64_t vs, bool full, PcgWork** out) {
    Solver* S;
    PC_TRY(solver_get(g, &S));
    PcgWork& w = S->pcg[dtype == PC_C64 ? 0 : 1];
    const int64_t esz = dtype == PC_C64 ? 8 : 16;
    // partial-sum slots: stencil CTAs, vector CTAs, unpack CTAs (x4 for full space)
    const int nap = std::max(apply_config_for(g, full, 1, dtype).ctas, apply_config_for(g, full, nsys, dtype).ctas);
    const int npm = std::max(std::max(nap, vec_ctas(vs)), 4 * precond_partials(g));
    if (w.cap >= nsys && w.vs == vs && w.npart_max >= npm && w.dtype == dtype) {
        *out = &w;
        return PC_OK;
    }
    w.release();
    w.dtype = dtype;
    w.vs = vs;
    w.npart_max = npm;
    const size_t vb = (size_t)nsys * vs * esz;
    PC_CUDA_TRY(cudaMalloc(&w.R, vb));
    PC_CUDA_TRY(cudaMalloc(&w.Z, vb));
    PC_CUDA_TRY(cudaMalloc(&w.P, vb));
    PC_CUDA_TRY(cudaMalloc(&w.Q, vb));
    PC_CUDA_TRY(cudaMalloc(&w.part, sizeof(double) * 4 * (size_t)nsys * npm));
    PC_CUDA_TRY(cudaMalloc(&w.sc, sizeof(PcgScal) * nsys));
    PC_CUDA_TRY(cudaMalloc(&w.done, sizeof(int) * nsys));
    PC_CUDA_TRY(cudaMalloc(&w.blocks, sizeof(int) * 4 * nsys));
    PC_CUDA_TRY(cudaMalloc(&w.kslots, sizeof(int) * 4 * nsys));
    PC_CUDA_TRY(cudaMallocHost(&w.h_sc, sizeof(PcgScal) * nsys));
    w.cap = nsys;
    *out = &w;
    return PC_OK;
}

template <typename C>
static int pcg_solve_t(pc_grid* g, int dtype, int nsys, const int* blocks, const int* kslots, double sigma,
                       const void* Bv, void* Xv, double tol, int maxit, PcgResult* res, cudaStream_t s, bool pre32) {
    const bool full = blocks[0] < 0;
    for (int i = 0; i < nsys; ++i)
        if ((blocks[i] < 0) != full) return fail(PC_EINVAL, "pcg: mixing full-space and block systems");
    bool multi_k = false;  // systems at Bloch slots other than 0
    for (int i = 0; kslots && i < nsys; ++i) {
        if (kslots[i] < 0 || kslots[i] >= g->nk) return fail(PC_EINVAL, "pcg: Bloch slot out of range");
        if (kslots[i] != 0) multi_k = true;
    }
    if (multi_k && !precond_multi_k(g)) return fail(PC_EINVAL, "pcg: several Bloch slots need the own DFT");
    const int64_t m = full ? g->n : g->nb;
    const int64_t vs = 3 * m;
    PcgWork* w;
    PC_TRY(pcg_work(g, dtype, nsys, vs, full, &w));
    const int npm = w->npart_max;
    double* part_a = w->part;                           // stencil <p,q> / ||b||^2
    double* part_b = w->part + (size_t)nsys * npm;      // ||r||^2
    double* part_c = w->part + (size_t)2 * nsys * npm;  // <r,z>
    // flexible CG when a complex128 solve is preconditioned in complex64: Re<r_new, z_old>
    const bool flex = pre32 && dtype == PC_C128;
    double* part_d = flex ? w->part + (size_t)3 * nsys * npm : nullptr;
    const C* B = static_cast<const C*>(Bv);
    C* X = static_cast<C*>(Xv);
    C* R = static_cast<C*>(w->R);
    C* Z = static_cast<C*>(w->Z);
    C* P = static_cast<C*>(w->P);
    C* Q = static_cast<C*>(w->Q);
    // block labels of the preconditioner subsystems
    std::vector<int> hb;
    if (full)
        for (int i = 0; i < nsys; ++i)
            for (int b = 0; b < 4; ++b) hb.push_back(b);
    else
        hb.assign(blocks, blocks + nsys);
    PC_CUDA_TRY(cudaMemcpyAsync(w->blocks, hb.data(), sizeof(int) * hb.size(), cudaMemcpyHostToDevice, s));
    std::vector<int> hk;  // Bloch slots of the preconditioner subsystems
    for (int i = 0; multi_k && i < nsys; ++i)
        for (int r = 0; r < (full ? 4 : 1); ++r) hk.push_back(kslots[i]);
    if (multi_k)
        PC_CUDA_TRY(cudaMemcpyAsync(w->kslots, hk.data(), sizeof(int) * hk.size(), cudaMemcpyHostToDevice, s));
    const int* d_sys_k = multi_k ? w->kslots : nullptr;
    const int vc = vec_ctas(vs);
    const dim3 vgrid(vc, nsys);

    // full-space preconditioning goes through the four block transforms
    void* Rb = nullptr;
    void* Zb = nullptr;
    if (full) {
        // reuse Q as gather buffer for r and the preconditioner workspace owner for z blocks
        PC_CUDA_TRY(cudaMallocAsync(&Rb, sizeof(C) * nsys * vs, s));
        PC_CUDA_TRY(cudaMallocAsync(&Zb, sizeof(C) * nsys * vs, s));
    }
    int nrz = 0;
    auto precondition = [&](const int* skip) -> int {
        if (!full) return precond_apply(g, dtype, nsys, R, Z, w->blocks, skip, sigma, s, part_c, &nrz, flex, d_sys_k);
        const int gb = (int)std::min<int64_t>((nsys * vs + 255) / 256, 16LL * device_sm_count());
        full_to_blocks<C><<<gb, 256, 0, s>>>(R, static_cast<C*>(Rb), g->N, nsys);
        note_launch();
        int np = 0;
        PC_TRY(precond_apply(g, dtype, 4 * nsys, Rb, Zb, w->blocks, nullptr, sigma, s, part_c, &np, flex, d_sys_k));
        nrz = 4 * np;  // the four block partials of a full system are contiguous
        blocks_to_full<C><<<gb, 256, 0, s>>>(static_cast<C*>(Zb), Z, g->N, nsys);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
        return PC_OK;
    };

    pcg_start<C><<<vgrid, 256, 0, s>>>(B, X, R, vs, part_a, npm);
    note_launch();
    pcg_start_bb<<<nsys, 256, 0, s>>>(w->sc, w->done, part_a, npm, vc, tol * tol);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());
    PC_TRY(precondition(full ? nullptr : w->done));
    pcg_start_rz<<<nsys, 256, 0, s>>>(w->sc, w->done, part_c, nrz);
    note_launch();
    pcg_copy<C><<<vgrid, 256, 0, s>>>(Z, P, vs, w->done);
    note_launch();
    PC_CUDA_TRY(cudaGetLastError());

    // stencil items: q_s = (A - sigma M) p_s with Re<p_s, q_s> partials in slot s
    std::vector<ApplyItem> items(nsys);
    for (int i = 0; i < nsys; ++i) {
        items[i].x = P + i * vs;
        items[i].y = Q + i * vs;
        items[i].mat = grid_mat(g, blocks[i]);
        items[i].shift = sigma;
        items[i].block = blocks[i];
        items[i].dot_slot = i;
        items[i].skip = w->done + i;
        items[i].kslot = kslots ? kslots[i] : 0;
    }
    const ApplyConfig cfg = apply_config_for(g, full, nsys, dtype);
    const int napc = cfg.ctas;
    const int chunk = 4;
    auto iterate = [&]() -> int {
        PC_TRY(grid_apply(g, dtype, full, items.data(), nsys, part_a, npm, s, &cfg));
        pcg_alpha<<<nsys, 256, 0, s>>>(w->sc, w->done, part_a, npm, napc);
        note_launch();
        pcg_update_xr<C><<<vgrid, 256, 0, s>>>(X, R, P, Q, w->sc, w->done, vs, part_b, npm, flex ? Z : nullptr,
                                                part_d);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
        PC_TRY(precondition(full ? nullptr : w->done));
        pcg_beta<<<nsys, 256, 0, s>>>(w->sc, w->done, part_b, npm, vc, part_c, nrz, maxit, part_d);
        note_launch();
        pcg_update_p<C><<<vgrid, 256, 0, s>>>(P, Z, w->sc, w->done, vs);
        note_launch();
        PC_CUDA_TRY(cudaGetLastError());
        return PC_OK;
    };
    // Chunks after the first (which creates the preconditioner workspace and FFT plans) replay
    // a CUDA graph of `chunk` iterations, captured once per (Bloch vector, systems, buffers,
    // shift); block systems on a non-default stream only.
    const bool graphs = !full && pcg_graphs_enabled() && s != nullptr && s != cudaStreamLegacy &&
                        s != cudaStreamPerThread;
    auto chunk_graph = [&]() -> int {
        std::vector<double> key = {(double)g->k.version, (double)g->kset_version, (double)dtype, (double)nsys, sigma,
                                   (double)maxit,
                                   (double)(uintptr_t)B, (double)(uintptr_t)X, (double)(uintptr_t)g->pre->d_work,
                                   (double)(uintptr_t)w->R, (double)(timing_enabled() ? 1 : 0), (double)npm,
                                   (double)flex, (double)(uintptr_t)g->d_split};  // the two-pass apply's scratch
        for (int i = 0; i < nsys; ++i) key.push_back((double)blocks[i]);
        for (int i = 0; i < nsys; ++i) key.push_back(kslots ? (double)kslots[i] : 0.0);
        if (w->gexec == nullptr || w->gkey != key) {
            w->drop_graph();
            cudaGraph_t graph = nullptr;
            PC_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const long long n0 = launch_count(), a0 = apply_launch_count();
            TimedSet* ts = timing_enabled() ? timing_capture_begin() : nullptr;
            int rc = PC_OK;
            for (int c = 0; c < chunk && rc == PC_OK; ++c) rc = iterate();
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (ts) timing_capture_end(ts);
            if (rc != PC_OK || e != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                timing_free(ts);
                return rc != PC_OK ? rc : cuda_fail(e, "cudaStreamEndCapture(pcg)");
            }
            e = cudaGraphInstantiate(&w->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                w->gexec = nullptr;
                timing_free(ts);
                return cuda_fail(e, "cudaGraphInstantiate(pcg)");
            }
            w->glaunches = launch_count() - n0;
            w->gapply = apply_launch_count() - a0;
            note_launch(-(int)w->glaunches);  // the capture launched nothing; replays are counted below
            note_apply_launch(-(int)w->gapply);
            w->gtimed = ts;
            w->gkey = key;
        }
        PC_CUDA_TRY(cudaGraphLaunch(w->gexec, s));
        note_launch((int)w->glaunches);
        note_apply_launch((int)w->gapply);
        return PC_OK;
    };
    int it = 0;
    bool all_done = false;
    while (!all_done) {
        if (graphs && it >= chunk) {
            PC_TRY(chunk_graph());
        } else {
            for (int c = 0; c < chunk; ++c) PC_TRY(iterate());
        }
        it += chunk;
        PC_CUDA_TRY(cudaMemcpyAsync(w->h_sc, w->sc, sizeof(PcgScal) * nsys, cudaMemcpyDeviceToHost, s));
        PC_CUDA_TRY(cudaStreamSynchronize(s));
        if (graphs && it > chunk && w->gtimed) timing_replayed(w->gtimed);
        all_done = true;
        for (int i = 0; i < nsys; ++i)
            if (!w->h_sc[i].done) all_done = false;
        if (it > maxit + chunk) break;  // the device loop stops by itself at maxit; host backstop
    }
    if (full) {
        cudaFreeAsync(Rb, s);
        cudaFreeAsync(Zb, s);
    }
    int worst = PC_OK;
    for (int i = 0; i < nsys; ++i) {
        const PcgScal& v = w->h_sc[i];
        res[i].iters = v.iters;
        res[i].status = v.done ? v.status : PC_ENOCONV;
        res[i].rel_resid = v.bb > 0 ? std::sqrt(v.rr / v.bb) : 0.0;
        if (res[i].status != PC_OK && worst == PC_OK) worst = res[i].status;
    }
    return PC_OK;
}

// One application of the reference-medium preconditioner outside a solve: block b (one system)
// or the full space (block < 0: gathered into its four blocks, each preconditioned, scattered
// back).  Scratch comes from the stream-ordered allocator and is released on the same stream.
template <typename C>
static int precond_once_t(pc_grid* g, int block, int dtype, bool fp32_inner, double sigma, const void* r, void* z,
                          cudaStream_t s) {
    struct Scratch {
        cudaStream_t s;
        void* p[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Scratch() {
            for (void* q : p)
                if (q) cudaFreeAsync(q, s);
        }
    } sc{s};
    const bool full = block < 0;
    const int nsys = full ? 4 : 1;
    const int64_t vs = 3 * g->nb;
    const bool lower = fp32_inner && dtype == PC_C128;
    int hb[4] = {0, 1, 2, 3};
    if (!full) hb[0] = block;
    PC_CUDA_TRY(cudaMallocAsync(&sc.p[0], sizeof(int) * 4, s));
    PC_CUDA_TRY(cudaMemcpyAsync(sc.p[0], hb, sizeof(int) * 4, cudaMemcpyHostToDevice, s));
    // the partial sums of Re<r, z> are not returned; they keep the unpack on the kernels a solve runs
    PC_CUDA_TRY(cudaMallocAsync(&sc.p[1], sizeof(double) * nsys * precond_partials(g), s));
    double* d_part = static_cast<double*>(sc.p[1]);
    const void* rin = r;
    void* zout = z;
    const int gb = (int)std::min<int64_t>((4 * g->nb + 255) / 256, 16LL * device_sm_count());
    if (full) {
        PC_CUDA_TRY(cudaMallocAsync(&sc.p[2], sizeof(C) * 4 * vs, s));
        PC_CUDA_TRY(cudaMallocAsync(&sc.p[3], sizeof(C) * 4 * vs, s));
        full_to_blocks<C><<<gb, 256, 0, s>>>(static_cast<const C*>(r), static_cast<C*>(sc.p[2]), g->N, 1);
        note_launch();
        rin = sc.p[2];
        zout = sc.p[3];
    }
    PC_TRY(precond_apply(g, dtype, nsys, rin, zout, static_cast<const int*>(sc.p[0]), nullptr, sigma, s, d_part,
                         nullptr, lower));
    if (full) {
        blocks_to_full<C><<<gb, 256, 0, s>>>(static_cast<const C*>(sc.p[3]), static_cast<C*>(z), g->N, 1);
        note_launch();
    }
    PC_CUDA_TRY(cudaGetLastError());
    return PC_OK;
}

int precond_once(pc_grid* g, int block, int dtype, bool fp32_inner, double sigma, const void* r, void* z,
                 cudaStream_t s) {
    if (dtype == PC_C64) return precond_once_t<float2>(g, block, dtype, false, sigma, r, z, s);
    return precond_once_t<double2>(g, block, dtype, fp32_inner, sigma, r, z, s);
}

int pcg_solve(pc_grid* g, int dtype, int nsys, const int* blocks, double sigma, const void* B, void* X, double tol,
              int maxit, PcgResult* res, cudaStream_t s, bool pre32, const int* kslots) {
    if (nsys <= 0) return PC_OK;
    if (!g->k.set) return fail(PC_ESTATE, "pcg: call pc_set_k first");
    if (!(tol > 0) || maxit < 1) return fail(PC_EINVAL, "pcg: tol must be > 0 and maxit >= 1");
    if (dtype == PC_C64)
        return pcg_solve_t<float2>(g, dtype, nsys, blocks, kslots, sigma, B, X, tol, maxit, res, s, false);
    return pcg_solve_t<double2>(g, dtype, nsys, blocks, kslots, sigma, B, X, tol, maxit, res, s, pre32);
}

}  // namespace pc

Solver::~Solver() {
    pcg[0].release();
    pcg[1].release();
}
