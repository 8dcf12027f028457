// Autotuner of the stencil-apply launch: for one grid layout (extents, precision, parity blocks
// or full space, material kind, lattice) and one batch size, time every applicable kernel and
// launch shape on the GPU and keep the fastest.
//
// Candidates: the plane-pipelined and row-tile kernels (complex64 blocks) with several persistent
// CTA counts, the
// TMA tile kernel (16-wide and 8-wide tiles) and the register-staged kernel (four tile shapes),
// each with k-chunkings that target one, two or four resident CTAs per SM.  Results live in a
// process-wide table keyed by (X, Y, Z, dtype, layout, material kind, lattice, batch-size
// bucket, SM count) and, when PC_TUNE_CACHE names a file, are read from and appended to it
// (one JSON object per key), so a later process starts tuned.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "pc_internal.h"
#include "pc_solver.h"

namespace pc {

namespace {

std::mutex g_tune_mu;
std::map<std::string, ApplyConfig> g_tuned;
bool g_loaded = false;

int bucket_of(int nitems) {
    int b = 1;
    while (b < nitems && b < 64) b <<= 1;
    return b;
}

std::string tune_key(int X, int Y, int Z, int dtype, bool full, int matkind, bool cubic, int nitems) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "%d,%d,%d,%s,%s,%s,%s,n%d,sm%d", X, Y, Z, dtype == PC_C64 ? "c64" : "c128",
                  full ? "full" : "blocks", matkind == 2 ? "nodewise" : (matkind ? "theta" : "phase"),
                  cubic ? "cubic" : "general",
                  bucket_of(nitems), device_sm_count());
    return buf;
}

const char* cache_path() {
    const char* p = std::getenv("PC_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

// One entry per line:  "key": {"kind": K, "shape": S, "tz": T, "ctas": C}
void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = cache_path();
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        const size_t q0 = line.find('"'), q1 = line.find('"', q0 + 1);
        if (q0 == std::string::npos || q1 == std::string::npos) continue;
        const std::string key = line.substr(q0 + 1, q1 - q0 - 1);
        int kind = -1, shape = 0, tz = 0, ctas = 0;
        if (std::sscanf(line.c_str() + q1 + 1, " : {\"kind\": %d, \"shape\": %d, \"tz\": %d, \"ctas\": %d", &kind, &shape,
                        &tz, &ctas) != 4)
            continue;
        if (kind < 0 || kind > 4 || ctas < 1) continue;
        ApplyConfig c;
        c.shape = shape;
        c.tz = tz;
        c.ctas = ctas;
        c.tma = kind == 1;
        c.row = kind == 2;
        c.split = kind == 3;
        c.pipe = kind == 4;
        g_tuned[key] = c;
    }
}

void append_locked(const std::string& key, const ApplyConfig& c, double us) {
    const char* path = cache_path();
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    if (!f) return;
    f << "\"" << key << "\": {\"kind\": " << config_kind(c) << ", \"shape\": " << c.shape
      << ", \"tz\": " << c.tz << ", \"ctas\": " << c.ctas << ", \"us\": " << us << "}\n";
}

}  // namespace

bool tuned_config(int X, int Y, int Z, int dtype, bool full, int matkind, bool cubic, int nitems, ApplyConfig* out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_locked();
    auto it = g_tuned.find(tune_key(X, Y, Z, dtype, full, matkind, cubic, nitems));
    if (it == g_tuned.end()) return false;
    *out = it->second;
    // a tuned chunking for a bucket is reused for every batch size in it: recount the CTAs
    if (out->split) {
        out->ctas = split_apply_ctas((int64_t)X * Y * Z);
    } else if (out->pipe) {
        out->ctas = pipe_apply_ctas(X, Y, Z, matkind, nitems, out->tz);
    } else if (out->row) {
        out->ctas = row_apply_ctas(X, Y, Z, matkind, nitems, out->tz);
    } else {
        const int tx = out->tma ? ((out->shape == 0) ? 16 : 8) : tile_tx(out->shape);
        const int ty = out->tma ? ((out->shape == 0 && dtype == PC_C64) ? 16 : 8) : tile_ty(out->shape);
        out->ctas = ((X + tx - 1) / tx) * ((Y + ty - 1) / ty) * ((Z + out->tz - 1) / out->tz);
    }
    return true;
}

ApplyConfig apply_config_for(const pc_grid* g, bool full, int nitems, int dtype) {
    const int X = full ? g->N : g->X, Y = full ? g->N : g->Y, Z = g->Z;
    ApplyConfig c;
    if (tuned_config(X, Y, Z, dtype, full, g->matkind, g->cubic, nitems, &c)) return c;
    return choose_apply_config(X, Y, Z, nitems, dtype, !full, g->matkind);
}

// Time one candidate on scratch vectors: after two warm-up launches, the best of three
// measurements of eight back-to-back launches (so that host enqueue time overlaps the GPU).
static int time_candidate(pc_grid* g, int dtype, bool full, std::vector<ApplyItem>& items, const ApplyConfig& c,
                          cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* us) {
    for (int rep = 0; rep < 2; ++rep)
        PC_TRY(grid_apply(g, dtype, full, items.data(), (int)items.size(), nullptr, 0, s, &c));
    float best = 1e30f;
    for (int m = 0; m < 3; ++m) {
        PC_CUDA_TRY(cudaEventRecord(e0, s));
        for (int rep = 0; rep < 8; ++rep)
            PC_TRY(grid_apply(g, dtype, full, items.data(), (int)items.size(), nullptr, 0, s, &c));
        PC_CUDA_TRY(cudaEventRecord(e1, s));
        PC_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms / 8.f);
    }
    *us = 1e3 * best;
    return PC_OK;
}

static std::vector<ApplyConfig> candidates(int X, int Y, int Z, int dtype, bool full, int matkind, int nitems) {
    std::vector<ApplyConfig> out;
    const int sm = device_sm_count();
    // two-pass kernels: the default for complex128; for complex64 a candidate while the batch's
    // scratch (15 complex64 flux arrays per extended cell plus x's ghost cells) fits in L2
    // (126 MB on GB300)
    const double split_mb = (double)split_scratch_bytes(X, Y, Z, nitems, dtype) / (1 << 20);
    if (matkind == 2) {  // a nodewise material: the complex128 two-pass kernels only
        if (dtype == PC_C128) {
            ApplyConfig c;
            c.split = true;
            c.tz = Z;
            c.ctas = split_apply_ctas((int64_t)X * Y * Z);
            out.push_back(c);
        }
        return out;
    }
    if (dtype == PC_C128 || split_mb <= 96.0) {
        ApplyConfig c;
        c.split = true;
        c.tma = false;
        c.shape = 0;
        c.tz = Z;
        c.ctas = split_apply_ctas((int64_t)X * Y * Z);
        out.push_back(c);
    }
    auto chunkings = [&](int tiles, int per_sm, ApplyConfig base, int minplanes) {
        const long target = (long)sm * per_sm;
        long nch = (target + (long)tiles * nitems - 1) / ((long)tiles * nitems);
        const long maxch = std::max(1, Z / minplanes);
        nch = std::max(1L, std::min(nch, maxch));
        base.tz = (int)((Z + nch - 1) / nch);
        base.ctas = tiles * ((Z + base.tz - 1) / base.tz);
        for (auto& o : out)
            if (!o.pipe && o.row == base.row && o.tma == base.tma && o.shape == base.shape && o.tz == base.tz) return;
        out.push_back(base);
    };
    if (!full && dtype == PC_C64 && pipe_geom_ok(X, Y, Z, matkind)) {
        for (int minseg : {4, 8, 12, 24, 48}) {
            ApplyConfig c;
            c.pipe = true;
            c.shape = 0;
            c.tz = minseg;
            c.ctas = pipe_apply_ctas(X, Y, Z, matkind, nitems, minseg);
            bool dup = false;
            for (auto& o : out) dup = dup || (o.pipe && o.ctas == c.ctas);
            if (!dup) out.push_back(c);
        }
    }
    if (!full && dtype == PC_C64 && X % 2 == 0 && row_geom_fits(X, Y, Z, matkind)) {
        for (int minseg : {4, 8, 12, 24, 48}) {
            ApplyConfig c;
            c.row = true;
            c.tma = false;
            c.shape = 0;
            c.tz = minseg;
            c.ctas = row_apply_ctas(X, Y, Z, matkind, nitems, minseg);
            bool dup = false;
            for (auto& o : out) dup = dup || (o.row && o.ctas == c.ctas);
            if (!dup) out.push_back(c);
        }
    }
    if (X % 2 == 0 && X >= 8 && Y >= 8) {
        for (int shape : {0, 1}) {
            const int tx = shape == 0 ? 16 : 8, ty = (shape == 0 && dtype == PC_C64) ? 16 : 8;
            const int tiles = ((X + tx - 1) / tx) * ((Y + ty - 1) / ty);
            for (int per_sm : {1, 2, 4}) {
                ApplyConfig c;
                c.tma = true;
                c.shape = shape;
                chunkings(tiles, per_sm, c, 6);
            }
        }
    }
    for (int shape = (dtype == PC_C128 ? 1 : 0); shape <= 3; ++shape) {
        if (X < tile_tx(shape) || Y < tile_ty(shape)) continue;
        const int tiles = ((X + tile_tx(shape) - 1) / tile_tx(shape)) * ((Y + tile_ty(shape) - 1) / tile_ty(shape));
        for (int per_sm : {2, 4, 8}) {
            ApplyConfig c;
            c.tma = false;
            c.shape = shape;
            chunkings(tiles, per_sm, c, 4);
        }
    }
    return out;
}

int autotune_layout(pc_grid* g, int dtype, bool full, int nitems, cudaStream_t s, int verbose) {
    const int X = full ? g->N : g->X, Y = full ? g->N : g->Y, Z = g->Z;
    const std::string key = tune_key(X, Y, Z, dtype, full, g->matkind, g->cubic, nitems);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_locked();
        if (g_tuned.count(key)) return PC_OK;
    }
    const int n = bucket_of(nitems);
    const int64_t m = full ? g->n : g->nb;
    const size_t vbytes = (size_t)3 * m * (dtype == PC_C64 ? 8 : 16);
    void* buf = nullptr;
    PC_CUDA_TRY(cudaMalloc(&buf, 2 * vbytes * n));
    cudaMemsetAsync(buf, 0, 2 * vbytes * n, s);
    std::vector<ApplyItem> items(n);
    for (int i = 0; i < n; ++i) {
        const int block = full ? -1 : (i & 3);
        items[i].x = static_cast<char*>(buf) + vbytes * i;
        items[i].y = static_cast<char*>(buf) + vbytes * (n + i);
        items[i].mat = grid_mat(g, block);
        items[i].shift = -1.0;
        items[i].block = block;
        items[i].dot_slot = -1;
        items[i].skip = nullptr;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ApplyConfig best;
    double best_us = 1e30;
    int rc = PC_OK;
    const bool was_timing = timing_enabled();
    if (was_timing) pc_stats_timing(0);  // candidate launches stay out of the apply statistics
    for (const ApplyConfig& c : candidates(X, Y, Z, dtype, full, g->matkind, n)) {
        double us = 0;
        rc = time_candidate(g, dtype, full, items, c, s, e0, e1, &us);
        if (rc != PC_OK) break;
        if (verbose)
            std::fprintf(stderr, "[pcband tune] %s kind=%s shape=%d tz=%d ctas=%d: %.1f us\n", key.c_str(),
                         c.pipe ? "pipe" : (c.split ? "split" : (c.row ? "row" : (c.tma ? "tma" : "regs"))), c.shape,
                         c.tz, c.ctas, us);
        if (us < best_us) {
            best_us = us;
            best = c;
        }
    }
    if (was_timing) pc_stats_timing(1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (rc != PC_OK) return rc;
    if (best_us < 1e30) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = best;
        append_locked(key, best, best_us);
    }
    return PC_OK;
}

}  // namespace pc

using namespace pc;

extern "C" int pc_autotune(pc_grid* g, int dtype, int layout, int nitems, void* stream) {
    if (!g) return fail(PC_EINVAL, "pc_autotune: null grid");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_autotune: dtype must be PC_C64 or PC_C128");
    if (layout < 0 || layout > 2) return fail(PC_EINVAL, "pc_autotune: layout must be 0 (blocks), 1 (full) or 2 (both)");
    if (nitems < 1 || nitems > 64) return fail(PC_EINVAL, "pc_autotune: nitems must be in 1..64");
    if (!g->k.set) return fail(PC_ESTATE, "pc_autotune: call pc_set_k first");
    cudaStream_t s = (cudaStream_t)stream;
    if (layout == 0 || layout == 2) PC_TRY(autotune_layout(g, dtype, false, nitems, s, 0));
    if (layout == 1 || layout == 2) PC_TRY(autotune_layout(g, dtype, true, nitems, s, 0));
    return PC_OK;
}

extern "C" int pc_tuned_config(const pc_grid* g, int dtype, int layout, int nitems, int* kind, int* shape, int* tz,
                               int* ctas) {
    if (!g || !kind || !shape || !tz || !ctas) return fail(PC_EINVAL, "pc_tuned_config: null argument");
    if (dtype != PC_C64 && dtype != PC_C128) return fail(PC_EINVAL, "pc_tuned_config: bad dtype");
    if (layout != 0 && layout != 1) return fail(PC_EINVAL, "pc_tuned_config: layout must be 0 or 1");
    const ApplyConfig c = apply_config_for(g, layout == 1, nitems < 1 ? 1 : nitems, dtype);
    *kind = config_kind(c);
    *shape = c.shape;
    *tz = c.tz;
    *ctas = c.ctas;
    return PC_OK;
}
