// Batched band solves: many Bloch vectors on several grids (ragged sizes) at once.
//
// Two levels.  On the device, pc_eigs_multi solves a chunk of Bloch vectors of one grid in
// lockstep: every (Bloch vector, parity block) pair is a space of the same Krylov-Schur
// iteration, and one stencil launch, one preconditioner launch and one Gram launch serve all
// unfinished spaces (each item of a launch carries its Bloch slot; the Fourier tables are per
// slot).  On the host, a pool of worker threads, each with its own CUDA stream and its own copy
// of the grid it is working on, takes (grid, chunk of Bloch vectors) items from a shared queue
// ordered largest grid first, so small grids fill the GPU next to large ones and no grid handle
// is ever used by two threads.  Chunks are sized so that a launch covers about 2^22 nodes of
// systems (small grids take many Bloch vectors per chunk, the largest one).  Launch shapes are
// tuned once per grid size before the workers start.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pc_internal.h"
#include "pc_solver.h"

using namespace pc;

extern "C" int pc_grid_clone(const pc_grid* src, pc_grid** out) {
    if (!src || !out) return fail(PC_EINVAL, "pc_grid_clone: null argument");
    *out = nullptr;
    pc_grid* g = new pc_grid();
    g->N = src->N;
    g->X = src->X;
    g->Y = src->Y;
    g->Z = src->Z;
    g->n = src->n;
    g->nb = src->nb;
    g->C0 = src->C0;
    g->rho0 = src->rho0;
    g->L = src->L;
    std::memcpy(g->Chat, src->Chat, sizeof(g->Chat));
    std::memcpy(g->rhohat, src->rhohat, sizeof(g->rhohat));
    std::memcpy(g->Ainv, src->Ainv, sizeof(g->Ainv));
    g->cubic = src->cubic;
    g->matkind = src->matkind;
    g->mean_theta = src->mean_theta;
    g->sigma_cmax = src->sigma_cmax;
    g->sigma_rmax = src->sigma_rmax;
    g->mat_pitch = src->mat_pitch;
    g->device = src->device;
    g->P64 = src->P64;
    g->P32 = src->P32;
    const size_t esz = g->matkind == 2 ? 22 * sizeof(double) : (g->matkind ? sizeof(float) : sizeof(uint8_t));
    auto dup = [&](const void* from, void** to, size_t bytes) -> int {
        if (!from) return PC_OK;
        PC_CUDA_TRY(cudaMalloc(to, bytes));
        PC_CUDA_TRY(cudaMemcpy(*to, from, bytes, cudaMemcpyDeviceToDevice));
        return PC_OK;
    };
    int rc = PC_OK;
    cudaError_t e = cudaMalloc(&g->d_err, sizeof(int));
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(error word)");
    if (rc == PC_OK) cudaMemset(g->d_err, 0, sizeof(int));
    if (rc == PC_OK) rc = dup(src->d_mat_full, &g->d_mat_full, g->n * esz);
    for (int b = 0; b < 4 && rc == PC_OK; ++b) rc = dup(src->d_mat_blk[b], &g->d_mat_blk[b], g->nb * esz);
    for (int b = 0; b < 4 && rc == PC_OK; ++b)
        rc = dup(src->d_mat_row[b], &g->d_mat_row[b], (size_t)g->mat_pitch * g->Y * g->Z * esz);
    if (rc != PC_OK) {
        pc_grid_destroy(g);
        return rc;
    }
    *out = g;
    return PC_OK;
}

extern "C" int pc_eigs_batch(pc_batch_job* jobs, int njobs, const pc_options* opt_in, int workers,
                             pc_batch_info* info) {
    if (!jobs || njobs < 1) return fail(PC_EINVAL, "pc_eigs_batch: no jobs");
    pc_options opt;
    if (opt_in) opt = *opt_in;
    else pc_options_default(&opt);
    int64_t total = 0;
    for (int j = 0; j < njobs; ++j) {
        const pc_batch_job& J = jobs[j];
        if (!J.grid || J.nk < 0 || (J.nk > 0 && (!J.kappas || !J.evals)) || J.nev < 1)
            return fail(PC_EINVAL, "pc_eigs_batch: job " + std::to_string(j) + " is incomplete");
        total += J.nk;
    }
    if (workers < 1) workers = 1;
    if (workers > 16) workers = 16;
    auto t0 = std::chrono::steady_clock::now();

    // work items (chunks of Bloch vectors of one grid), largest grids first (k order kept)
    struct Item {
        int job, k, nk;
    };
    const bool full = opt.full_space != 0;
    const int bs = std::max(1, std::min(opt.block_size, 16));
    const int nper = full ? 1 : 4;
    auto chunk_of = [&](const pc_grid* g) {
        const int64_t m = full ? g->n : g->nb;
        int64_t K = opt.kbatch > 0 ? opt.kbatch : ((int64_t)1 << 22) / std::max<int64_t>(1, (int64_t)bs * nper * m);
        K = std::max<int64_t>(1, std::min<int64_t>(K, opt.kbatch > 0 ? kMaxKSlots : 16));
        return (int)std::min<int64_t>(K, pc_eigs_multi_max(g));
    };
    std::vector<Item> items;
    for (int j = 0; j < njobs; ++j) {
        const int K = chunk_of(jobs[j].grid);
        for (int k = 0; k < jobs[j].nk; k += K) items.push_back({j, k, std::min(K, jobs[j].nk - k)});
    }
    std::stable_sort(items.begin(), items.end(),
                     [&](const Item& a, const Item& b) { return jobs[a.job].grid->n > jobs[b.job].grid->n; });

    // tune the launch shapes of every grid size once, before the workers compete for the GPU
    if (workers > (int)items.size()) workers = (int)std::max<size_t>(1, items.size());
    if (opt.autotune) {
        for (int j = 0; j < njobs; ++j) {
            if (jobs[j].nk == 0) continue;
            pc_grid* g = jobs[j].grid;
            PC_TRY(pc_set_k(g, jobs[j].kappas));
            const int nsys = bs * nper * std::min(chunk_of(g), jobs[j].nk);
            const bool mixed = opt.precision == PC_PREC_MIXED;
            PC_TRY(autotune_layout(g, mixed ? PC_C64 : PC_C128, full, nsys, (cudaStream_t)opt.stream, 0));
            if (mixed) PC_TRY(autotune_layout(g, PC_C128, full, nsys, (cudaStream_t)opt.stream, 0));
        }
        if (opt.stream) cudaStreamSynchronize((cudaStream_t)opt.stream);
        opt.autotune = 0;
    }
    if (opt.stream) cudaStreamSynchronize((cudaStream_t)opt.stream);

    std::atomic<size_t> next{0};
    std::atomic<int> failed{0}, hard{PC_OK};
    std::atomic<long long> pcg{0};
    std::mutex mu;
    double max_res = 0.0;
    std::string first_msg;  // error text of the first failed solve (error text is per thread)
    int dev = 0;
    cudaGetDevice(&dev);

    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            hard = PC_ECUDA;
            return;
        }
        pc_options o = opt;
        o.stream = s;
        int cur_job = -1;
        pc_grid* clone = nullptr;
        for (;;) {
            if (hard.load() != PC_OK) break;
            const size_t i = next.fetch_add(1);
            if (i >= items.size()) break;
            const Item it = items[i];
            const pc_batch_job& J = jobs[it.job];
            if (it.job != cur_job) {
                if (clone) pc_grid_destroy(clone);
                clone = nullptr;
                if (pc_grid_clone(J.grid, &clone) != PC_OK) {
                    hard = PC_ENOMEM;
                    break;
                }
                cur_job = it.job;
            }
            std::vector<pc_eigs_info> inf(it.nk);
            std::memset(inf.data(), 0, sizeof(pc_eigs_info) * it.nk);
            int rc = pc_eigs_multi(clone, it.nk, J.kappas + 3 * it.k, J.nev, J.sigma, &o,
                                   J.evals + (size_t)it.k * J.nev, nullptr,
                                   J.block_of ? J.block_of + (size_t)it.k * J.nev : nullptr, inf.data());
            const bool soft = rc == PC_OK || rc == PC_ENOCONV;  // per Bloch vector statuses are valid
            int nfail = 0;
            for (int q = 0; q < it.nk; ++q) {
                const int st = soft ? inf[q].status : rc;
                if (J.status) J.status[it.k + q] = st;
                if (st != PC_OK) ++nfail;
            }
            if (rc != PC_OK) {
                failed.fetch_add(nfail);
                std::lock_guard<std::mutex> lk(mu);
                if (first_msg.empty()) first_msg = pc_last_error();
                if (rc != PC_ENOCONV && rc != PC_EBREAKDOWN) hard = rc;
            }
            pcg.fetch_add(inf[0].pcg_iters);
            std::lock_guard<std::mutex> lk(mu);
            for (int q = 0; q < it.nk; ++q)
                if (std::isfinite(inf[q].max_rel_resid)) max_res = std::max(max_res, inf[q].max_rel_resid);
        }
        if (clone) pc_grid_destroy(clone);
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w) pool.emplace_back(worker);
    for (auto& t : pool) t.join();

    if (info) {
        info->workers = workers;
        info->kpoints = (int)total;
        info->failed = failed.load();
        info->pcg_iters = pcg.load();
        info->max_rel_resid = max_res;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (hard.load() != PC_OK) return fail(hard.load(), "pc_eigs_batch: a solve failed: " + first_msg);
    return failed.load() ? fail(PC_ENOCONV, "pc_eigs_batch: " + std::to_string(failed.load()) +
                                                " Bloch vectors did not converge (see status): " + first_msg)
                         : PC_OK;
}
