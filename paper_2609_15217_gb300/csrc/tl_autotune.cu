// tl_autotune.cu -- the size-aware dispatcher of the C ABI: per n, which
// kernel variant (thread-to-system mapping and storage) and block size each
// operation launches.  The paper reports "best X" curves where a run-time
// dispatcher picks, at each problem size, the fastest specialization of a
// solver family (Sec. 4.1, reporting convention); tl_autotune builds that
// table by timing every registered variant on the current device, and
// tl_dispatch_set / tl_dispatch_get read and write it directly.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "tinylu.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_persist_sizes.h"
#include "tl_smem.cuh"

namespace tl {
namespace {

// Uniform [-1, 1) numbers from a 64-bit counter hash (splitmix64 finalizer),
// so the tuning batch needs no host data.
__global__ void k_fill_uniform(double *p, int64_t count, uint64_t seed)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint64_t z = seed + static_cast<uint64_t>(i) * 0x9e3779b97f4a7c15ULL;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        p[i] = static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
}

bool op_takes_variant(int op) { return op == kOpGesv || op == kOpGesvLU || op == kOpGetrf; }

// A size refines only when refinement beat binary64 by this factor on the
// tuning batch.  The batch is uniform [-1, 1] (well conditioned: every
// system refines); on ill-conditioned systems refinement falls back and pays
// for both solves, so a tie on the tuning batch is a loss on such data
// (measured on the benchmark's ragged mix, half of it kappa in [1e2, 1e8]:
// refining n = 12 and 19, 1-4% faster on the tuning batch, made the mix 5%
// slower).
constexpr float kRefineMargin = 0.85f;

// Timed runs per candidate: the first warms up, the fastest of the others
// counts.  With 2 timed runs the choice between variants within 1-3% of
// each other changed from one bench run to the next; 4 narrow that noise.
constexpr int kTuneReps = 5;

// The choice of tl_gesv_batched / tl_getrf_batched for (n, layout), and for
// tl_getrs_batched the register kernel with the same lane count when there
// is one.  The ragged solves keep their own table (tl_autotune_ragged).
void set_gesv_family(tl_handle *h, int n, int layout, int variant, int block)
{
    for (int op = 0; op < kOps; ++op)
        if (op_takes_variant(op)) h->choice[n][layout][op] = Choice{variant, block};
    const int lanes = variant % 100;
    const VariantList &lo = registry(n, layout, kOpGetrs);
    for (int i = 0; i < lo.count; ++i)
        if (lo.v[i].kind == 0 && lo.v[i].lanes == lanes) h->choice[n][layout][kOpGetrs] = Choice{lanes, 0};
}

// Tuning batch for size n: about 1.6 GFLOP of algorithmic work (some 2 ms at
// the rates these kernels reach), never fewer than 512 systems per SM nor
// more than 2^19: the shared-memory variants only show their speed once
// every SM holds several waves of their blocks.
int64_t tuning_batch(const tl_handle *h, int n)
{
    const double fl = 2.0 * ((n - 1.0) * n * (2.0 * n - 1.0) / 6.0 + n * (n - 1.0)) + n * (n - 1.0) / 2.0 + 2.0 * n;
    int64_t b = static_cast<int64_t>(1.6e9 / fl);
    const int64_t lo = static_cast<int64_t>(h->sm_count) * 512;
    b = b < lo ? lo : b;
    return b > (int64_t(1) << 19) ? (int64_t(1) << 19) : b;
}

// Homogeneous ragged batch for the tuner: every system of size n, stored
// one after another.
__global__ void k_ragged_layout(int64_t S, int n, int32_t *nv, int64_t *a_off, int64_t *b_off)
{
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < S;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        nv[s] = n;
        a_off[s] = s * n * n;
        b_off[s] = s * n;
    }
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" tl_status tl_dispatch_set(tl_handle *h, int n, tl_layout layout, int variant, int block)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 3);
    if (block != 0 && block != 32 && block != 64 && block != 128) return fail_arg(h, 5);
    if (variant == 0) {
        for (int op = 0; op < kOps; ++op) h->choice[n][layout][op] = Choice{0, 0};
        return TL_OK;
    }
    bool found = false;
    const VariantList &l = registry(n, layout, kOpGesv);
    for (int i = 0; i < l.count; ++i)
        if (variant_id(l.v[i].lanes, l.v[i].kind) == variant) found = true;
    if (!found) return fail_arg(h, 4);
    set_gesv_family(h, n, layout, variant, block);
    // the ragged kernels (binary64 and mixed precision): the register kernel
    // with the same lane count, or the shared-memory kernel of the same id,
    // when there is one
    const int lanes = variant % 100;
    for (int op : {static_cast<int>(kOpRagged), static_cast<int>(kOpRaggedIr)}) {
        const VariantList &lo = registry(n, layout, op);
        for (int i = 0; i < lo.count; ++i)
            if (lo.v[i].kind == 0 && lo.v[i].lanes == lanes) h->choice[n][layout][op] = Choice{lanes, 0};
        // the ragged solves also have shared-memory kernels (per-system slot)
        if ((op == kOpRagged || op == kOpRaggedIr) && variant >= 100) {
            const VariantList &lr = registry(n, kPerSystem, op);
            for (int i = 0; i < lr.count; ++i)
                if (variant_id(lr.v[i].lanes, lr.v[i].kind) == variant)
                    h->choice[n][kPerSystem][op] = Choice{variant, 0};
        }
    }
    return TL_OK;
}

extern "C" tl_status tl_dispatch_get(tl_handle *h, int n, tl_layout layout, int *variant, int *block)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n < 1 || n > TL_MAX_N) return fail_arg(h, 2);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 3);
    if (!variant) return fail_arg(h, 4);
    const Choice &c = h->choice[n][layout][kOpGesv];
    const Variant *v = find_variant(n, layout, kOpGesv, c.lanes ? c.lanes : default_lanes(n));
    *variant = v ? variant_id(v->lanes, v->kind) : 0;
    if (block) *block = c.block;
    return TL_OK;
}

extern "C" tl_status tl_autotune(tl_handle *h, int n_min, int n_max, tl_layout layout, const char *table_path)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n_min < 1 || n_min > TL_MAX_N) return fail_arg(h, 2);
    if (n_max < n_min || n_max > TL_MAX_N) return fail_arg(h, 3);
    if (layout != TL_LAYOUT_PER_SYSTEM && layout != TL_LAYOUT_INTERLEAVED) return fail_arg(h, 4);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(nullptr, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return TL_ERR_UNSUPPORTED;
    cudaGetLastError();

    auto batch_of = [&](int n) { return tuning_batch(h, n); };
    int64_t nA = 0, nv = 0, batch = 0;
    for (int n = n_min; n <= n_max; ++n) {
        const int64_t b = batch_of(n), l = (b + 31) / 32 * 32;
        nA = std::max<int64_t>(nA, static_cast<int64_t>(n) * n * l);
        nv = std::max<int64_t>(nv, static_cast<int64_t>(n) * l);
        batch = std::max(batch, b);
    }
    double *dA = nullptr, *db = nullptr, *dx = nullptr;
    int32_t *dp = nullptr, *di = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t ts = nullptr;  // a private non-blocking stream: nothing else is serialized behind the tuning
    tl_status st = TL_OK;
    struct Row {
        int n, variant, block;
        float ms;
    };
    std::vector<Row> table;
    auto cleanup = [&]() {
        cudaFree(dA);
        cudaFree(db);
        cudaFree(dx);
        cudaFree(dp);
        cudaFree(di);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ts) {
            cudaStreamSynchronize(ts);
            cudaStreamDestroy(ts);
        }
    };
    if (cudaMalloc(&dA, nA * sizeof(double)) != cudaSuccess || cudaMalloc(&db, nv * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dx, nv * sizeof(double)) != cudaSuccess || cudaMalloc(&dp, nv * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&di, batch * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return TL_ERR_NO_MEMORY;
    }
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        const tl_status fs = fail_cuda(h, cudaGetLastError());
        cleanup();
        return fs;
    }
    k_fill_uniform<<<h->sm_count * 4, 256, 0, ts>>>(dA, nA, 12345);
    k_fill_uniform<<<h->sm_count * 4, 256, 0, ts>>>(db, nv, 54321);

    for (int n = n_min; n <= n_max && st == TL_OK; ++n) {
        const int64_t bn = batch_of(n), ld = (bn + 31) / 32 * 32;
        SolveArgs args{dA, nullptr, db, dx, dp, di, ld, bn, 1};
        const VariantList &l = registry(n, layout, kOpGesv);
        float best_ms = 1e30f;
        int best_var = 0, best_block = 0;
        for (int i = 0; i < l.count && st == TL_OK; ++i) {
            const Variant *v = &l.v[i];
            for (int block : {32, 64, 128}) {
                if (block < v->lanes) continue;
                if (v->kind >= 1 && (block / v->lanes) * smem_sys_bytes(n, v->lanes) + 1024 > static_cast<size_t>(h->max_smem_per_block))
                    continue;
                float ms_best = 1e30f;
                for (int rep = 0; rep < kTuneReps; ++rep) {
                    cudaEventRecord(e0, ts);
                    st = launch_variant(h, v, n, block, args, ts);
                    cudaEventRecord(e1, ts);
                    if (st != TL_OK) break;
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        st = fail_cuda(h, cudaGetLastError());
                        break;
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0 && ms < ms_best) ms_best = ms;  // first run warms up
                }
                if (st != TL_OK) break;
                if (ms_best < best_ms) {
                    best_ms = ms_best;
                    best_var = variant_id(v->lanes, v->kind);
                    best_block = block;
                }
            }
        }
        if (st == TL_OK && best_var) {
            set_gesv_family(h, n, layout, best_var, best_block);
            table.push_back(Row{n, best_var, best_block, best_ms});
        }
    }
    cleanup();
    if (st == TL_OK && table_path) {
        FILE *f = std::fopen(table_path, "w");
        if (!f) return TL_ERR_INVALID_ARG;
        std::fprintf(f, "{\"layout\": %d, \"max_batch\": %lld, \"entries\": [", static_cast<int>(layout),
                     static_cast<long long>(batch));
        for (size_t i = 0; i < table.size(); ++i)
            std::fprintf(f, "%s{\"n\": %d, \"variant\": %d, \"lanes\": %d, \"storage\": \"%s\", \"block\": %d, "
                            "\"batch\": %lld, \"ms\": %.6f}",
                         i ? ", " : "", table[i].n, table[i].variant, table[i].variant % 100,
                         table[i].variant >= 100 ? "shared" : "registers", table[i].block,
                         static_cast<long long>(batch_of(table[i].n)), table[i].ms);
        std::fprintf(f, "]}\n");
        std::fclose(f);
    }
    return st;
}

extern "C" tl_status tl_autotune_ragged(tl_handle *h, int n_min, int n_max, const char *table_path)
{
    if (!h) return TL_ERR_INVALID_ARG;
    h->last_bad_arg = 0;
    if (n_min < 1 || n_min > TL_MAX_N) return fail_arg(h, 2);
    if (n_max < n_min || n_max > TL_MAX_N) return fail_arg(h, 3);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(nullptr, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return TL_ERR_UNSUPPORTED;
    cudaGetLastError();
    int64_t maxS = 0, maxA = 0, maxV = 0;
    for (int n = n_min; n <= n_max; ++n) {
        const int64_t S = tuning_batch(h, n);
        maxS = std::max(maxS, S);
        maxA = std::max(maxA, S * n * n);
        maxV = std::max(maxV, S * n);
    }
    double *dA = nullptr, *db = nullptr, *dx = nullptr;
    int32_t *dp = nullptr, *di = nullptr, *dref = nullptr, *dn = nullptr, *ws = nullptr;
    int64_t *da = nullptr, *dbo = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t ts = nullptr;
    auto cleanup = [&]() {
        if (ts) cudaStreamSynchronize(ts);
        for (void *p : {static_cast<void *>(dA), static_cast<void *>(db), static_cast<void *>(dx),
                        static_cast<void *>(dp), static_cast<void *>(di), static_cast<void *>(dref),
                        static_cast<void *>(dn), static_cast<void *>(ws), static_cast<void *>(da),
                        static_cast<void *>(dbo)})
            cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ts) cudaStreamDestroy(ts);
    };
    if (cudaMalloc(&dA, maxA * 8) != cudaSuccess || cudaMalloc(&db, maxV * 8) != cudaSuccess ||
        cudaMalloc(&dx, maxV * 8) != cudaSuccess || cudaMalloc(&dp, maxV * 4) != cudaSuccess ||
        cudaMalloc(&di, maxS * 4) != cudaSuccess || cudaMalloc(&dref, maxS * 4) != cudaSuccess ||
        cudaMalloc(&dn, maxS * 4) != cudaSuccess || cudaMalloc(&da, maxS * 8) != cudaSuccess ||
        cudaMalloc(&dbo, maxS * 8) != cudaSuccess ||
        cudaMalloc(&ws, ragged_ws_ints(maxS, true) * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return TL_ERR_NO_MEMORY;
    }
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        const tl_status fs = fail_cuda(h, cudaGetLastError());
        cleanup();
        return fs;
    }
    k_fill_uniform<<<h->sm_count * 4, 256, 0, ts>>>(dA, maxA, 2468);
    k_fill_uniform<<<h->sm_count * 4, 256, 0, ts>>>(db, maxV, 1357);

    // keep the caller's settings; while a size is tuned every other size
    // runs with a full warp per system (the smallest shared-memory slice),
    // so the slice of the launch is the tuned size's own
    const int mode = h->ragged_mode;
    h->ragged_mode = TL_RAGGED_PERSISTENT;
    Choice saved[TL_MAX_N + 1], saved_ir[TL_MAX_N + 1];
    signed char saved_route[TL_MAX_N + 1];
    for (int n = 1; n <= TL_MAX_N; ++n) {
        saved[n] = h->choice[n][kPerSystem][kOpRagged];
        saved_ir[n] = h->choice[n][kPerSystem][kOpRaggedIr];
        saved_route[n] = h->mixed_route[n];
        h->choice[n][kPerSystem][kOpRagged] = Choice{variant_id(n <= kPersistRegMaxN ? 1 : 32, 1), 0};
    }
    struct Row {
        int n, lanes, refine, ir_variant;
        float ms64, ms_mixed;
    };
    std::vector<Row> table;
    tl_status st = TL_OK;
    for (int n = n_min; n <= n_max && st == TL_OK; ++n) {
        const int64_t S = tuning_batch(h, n);
        k_ragged_layout<<<h->sm_count * 4, 256, 0, ts>>>(S, n, dn, da, dbo);
        RaggedArgs r{nullptr, nullptr, da, dA, dbo, db, dx, dbo, dp, di};
        auto time_it = [&](bool mixed, float *out) -> tl_status {
            RaggedArgs rr = r;
            rr.refine = mixed ? dref : nullptr;
            float best = 1e30f;
            for (int rep = 0; rep < kTuneReps; ++rep) {
                cudaEventRecord(e0, ts);
                const tl_status s2 = ragged_solve(h, S, dn, rr, ws, ts, mixed);
                cudaEventRecord(e1, ts);
                if (s2 != TL_OK) return s2;
                if (cudaEventSynchronize(e1) != cudaSuccess) return fail_cuda(h, cudaGetLastError());
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && ms < best) best = ms;  // the first run warms up
            }
            *out = best;
            return TL_OK;
        };
        int best_T = 0;
        float best64 = 1e30f;
        {
            for (int T : {1, 2, 4, 8, 16, 32}) {
                if (T == 1 && n > kPersistRegMaxN) continue;  // one thread in registers: small n only
                // only choices within the launch's slice: a larger one would
                // shrink the resident warps of every size in a mixed batch
                if (persist_need(n, T) > kPersistSliceDoubles) continue;
                h->choice[n][kPerSystem][kOpRagged] = Choice{variant_id(T, 1), 0};
                float ms = 0.f;
                if ((st = time_it(false, &ms)) != TL_OK) break;
                if (ms < best64) {
                    best64 = ms;
                    best_T = T;
                }
            }
            if (st != TL_OK) break;
            h->choice[n][kPerSystem][kOpRagged] = Choice{variant_id(best_T, 1), 0};
        }
        // mixed precision: every refinement kernel built for n (the
        // register kernel of its lane count, the shared-memory warp kernel)
        h->mixed_route[n] = 0;  // refine
        float ms_mixed = 1e30f;
        int best_ir = 0;
        const VariantList &li = registry(n, kPerSystem, kOpRaggedIr);
        for (int i = 0; i < li.count && st == TL_OK; ++i) {
            const int id = variant_id(li.v[i].lanes, li.v[i].kind);
            h->choice[n][kPerSystem][kOpRaggedIr] = Choice{id, 0};
            float ms = 0.f;
            if ((st = time_it(true, &ms)) != TL_OK) break;
            if (ms < ms_mixed) {
                ms_mixed = ms;
                best_ir = id;
            }
        }
        if (st != TL_OK) break;
        h->choice[n][kPerSystem][kOpRaggedIr] = saved_ir[n];
        h->mixed_route[n] = saved_route[n];
        // back to the neutral choice while the other sizes are tuned (the
        // winners are applied together at the end)
        h->choice[n][kPerSystem][kOpRagged] = Choice{variant_id(n <= kPersistRegMaxN ? 1 : 32, 1), 0};
        table.push_back(Row{n, best_T, ms_mixed < kRefineMargin * best64 ? 1 : 0, best_ir, best64, ms_mixed});
    }
    for (int n = 1; n <= TL_MAX_N; ++n) {
        h->choice[n][kPerSystem][kOpRagged] = saved[n];
        h->choice[n][kPerSystem][kOpRaggedIr] = saved_ir[n];
        h->mixed_route[n] = saved_route[n];
    }
    h->ragged_mode = mode;
    cleanup();
    if (st != TL_OK) return st;
    for (const Row &row : table) {
        if (row.lanes) h->choice[row.n][kPerSystem][kOpRagged] = Choice{variant_id(row.lanes, 1), 0};
        if (row.ir_variant) h->choice[row.n][kPerSystem][kOpRaggedIr] = Choice{row.ir_variant, 0};
        h->mixed_route[row.n] = static_cast<signed char>(row.refine ? 0 : 1);
    }
    if (table_path) {
        FILE *f = std::fopen(table_path, "w");
        if (!f) return TL_ERR_INVALID_ARG;
        std::fprintf(f, "{\"entries\": [");
        for (size_t i = 0; i < table.size(); ++i)
            std::fprintf(f, "%s{\"n\": %d, \"lanes\": %d, \"mixed_refines\": %d, \"ir_variant\": %d, "
                            "\"batch\": %lld, \"ms_fp64\": %.6f, \"ms_mixed\": %.6f}",
                         i ? ", " : "", table[i].n, table[i].lanes, table[i].refine, table[i].ir_variant,
                         static_cast<long long>(tuning_batch(h, table[i].n)), table[i].ms64, table[i].ms_mixed);
        std::fprintf(f, "]}\n");
        std::fclose(f);
    }
    return TL_OK;
}
