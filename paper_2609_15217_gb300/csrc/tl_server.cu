// tl_server.cu -- the request server of tinylu.h: a native request loop
// (one host thread per server) doing continuous batching of Newton and
// solve requests on one device.
//
// Life of a request: submit (descriptor copied, queued FIFO) -> admitted
// into a tick when a slot (stream) is free and the arena has room -> its
// inputs copied into its arena block, its points integrated by the fused
// Newton kernel of its law class (one launch per class over every request of
// the tick, through a job table) or its systems solved by one ragged LUpp
// over every solve of the tick -> results copied back to its host arrays ->
// done when its group's event completes (its arena block is released then;
// the tick's tables when the last group of the tick completes).
// Ticks on different slots overlap on the device; requests that arrive while
// ticks run wait at most until a slot frees up.
//
// There are no device-side waits: the request loop lives on the host, so a
// kernel never spins on a flag the host writes.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tinylu.h"
#include "tl_arena.h"
#include "tl_handle.h"
#include "tl_internal.h"
#include "tl_newton_types.h"

namespace tl {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int kMaxSlots = 16;
constexpr size_t kMaxJobsPerTick = 4096;

size_t up(size_t b) { return Arena::round_up(b); }

struct Req {
    int64_t id = 0;
    tl_request d{};
    NewtonJob job{};  // law parameters (Newton)
    Clock::time_point t_submit, t_done;
    bool done = false;
    int32_t status = TL_OK;
    size_t off = SIZE_MAX, bytes = 0;   // arena block
    size_t o_in = 0, o_x = 0, o_aux = 0, o_i1 = 0, o_i2 = 0;  // offsets inside the arena
    int fields() const { return d.law.id == TL_LAW_NORTON ? 12 : d.law.n * d.law.n + 2 * d.law.n; }
    int xrows() const { return d.law.id == TL_LAW_NORTON ? 7 : d.law.n; }
    bool has_aux() const { return d.kind == TL_REQ_NEWTON && d.law.id == TL_LAW_NORTON && d.aux; }
    // arena layout of the request's own buffers
    size_t layout(size_t base)
    {
        size_t o = base;
        const size_t c = static_cast<size_t>(d.count);
        if (d.kind == TL_REQ_NEWTON) {
            o_in = o; o += up(c * fields() * 8);
            o_x = o; o += up(c * xrows() * 8);
            o_aux = o; o += has_aux() ? up(c * 6 * 8) : 0;
            o_i1 = o; o += up(c * 4);
            o_i2 = o; o += up(c * 4);
        } else {
            const size_t n = static_cast<size_t>(d.n);
            o_in = o; o += up(c * n * n * 8);
            o_x = o; o += up(c * n * 8);   // b copied here, solved in place
            o_i1 = o; o += up(c * n * 4);
        }
        return o - base;
    }
    // tick-table bytes this request adds (job entry, or the ragged solve's
    // per-system arrays: n, a_off, b_off, piv_off, info)
    size_t table_bytes() const
    {
        return d.kind == TL_REQ_NEWTON ? sizeof(NewtonJob) : static_cast<size_t>(d.count) * 32;
    }
    int64_t systems() const { return d.kind == TL_REQ_SOLVE ? d.count : 0; }
};

// Requests of a tick that complete together: one Newton law class, all the
// solves, or the empty requests; `ev` (slot.evs[index]) is recorded after
// the group's results are copied back.
struct Group {
    std::vector<Req *> reqs;
    bool done = false;
    bool timed = false;  // kernel timing events recorded in kev[2g], kev[2g + 1]
};
constexpr int kMaxGroups = 2 * TL_MAX_N + 8;

// Bytes of a tick's scratch block: the tables plus the bucket workspace of
// the ragged solve over its `nsys` systems (so no tick ever grows a
// workspace with cudaMalloc or synchronizes the device).
size_t tick_scratch_bytes(size_t table, int64_t nsys)
{
    return table + (nsys > 0 ? up(ragged_ws_ints(nsys, false) * sizeof(int32_t)) : 0) + 4 * Arena::kAlign;
}

// Each slot runs its ticks on three streams: copies in (s_in), kernels
// (stream) and copies out (s_out), so that a tick's later classes copy
// their inputs while its earlier classes compute, and results go home while
// the next class runs.
struct Slot {
    cudaStream_t stream = nullptr;   // kernels
    cudaStream_t s_in = nullptr;     // host -> device copies
    cudaStream_t s_out = nullptr;    // device -> host copies
    std::vector<cudaEvent_t> evs;    // kMaxGroups events: group done (on s_out)
    std::vector<cudaEvent_t> ev_in;  // kMaxGroups: group inputs on the device (on s_in)
    std::vector<cudaEvent_t> ev_k;   // kMaxGroups: group kernels done (on stream)
    std::vector<cudaEvent_t> kev;  // 2 * kMaxGroups timing events around each group's kernels
    tl_handle *h = nullptr;  // own handle: the ragged solve's workspace is per handle
    bool busy = false;
    std::vector<Req *> reqs;
    std::vector<Group> groups;
    size_t scratch_off = SIZE_MAX, scratch_bytes = 0;
    char *stage = nullptr;  // page-locked staging of the tick tables
    size_t stage_bytes = 0;
};

}  // namespace
}  // namespace tl

using namespace tl;

struct tl_server {
    tl_handle *h = nullptr;
    int device = 0;
    tl_server_config cfg{};
    char *base = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<int64_t, Req *> reqs;
    int64_t next_id = 1;
    bool stop = false;
    bool paused = false;
    tl_server_stats stats{};
    std::thread loop;
    // kernel intervals (ms after t0_ev) of the completed groups
    cudaEvent_t t0_ev = nullptr;
    std::vector<std::pair<float, float>> kernel_spans;
    double busy_union();

    void run();
    bool form_tick(Slot &sl, std::vector<Req *> &batch, size_t &scratch_off, size_t &scratch_bytes);
    tl_status enqueue(Slot &sl, std::vector<Req *> &batch);
    void finish_group(Slot &sl, Group &g, int32_t status);
    void retire(Slot &sl, tl_status failed);
};

namespace {

tl_status check_request(const tl_request *r)
{
    if (!r) return TL_ERR_INVALID_ARG;
    if (r->count < 0) return TL_ERR_INVALID_ARG;
    if (r->kind == TL_REQ_NEWTON) {
        NewtonJob jb{};
        if (!law_params(r->law, &jb)) return TL_ERR_INVALID_ARG;
        if (r->count > 0 && (!r->in || !r->x || !r->i1 || !r->i2)) return TL_ERR_INVALID_ARG;
        if (r->ld_in != 0 && r->ld_in < r->count) return TL_ERR_INVALID_ARG;
        return TL_OK;
    }
    if (r->kind == TL_REQ_SOLVE) {
        if (r->n < 1 || r->n > TL_MAX_N) return TL_ERR_INVALID_ARG;
        if (r->count > 0 && (!r->in || !r->rhs || !r->x || !r->i1 || !r->i2)) return TL_ERR_INVALID_ARG;
        return TL_OK;
    }
    return TL_ERR_INVALID_ARG;
}

tl_status grow_stage(Slot &sl, size_t bytes)
{
    if (sl.stage_bytes >= bytes) return TL_OK;
    if (sl.stage) cudaFreeHost(sl.stage);
    sl.stage = nullptr;
    sl.stage_bytes = 0;
    const size_t want = std::max(bytes, static_cast<size_t>(1) << 20);
    if (cudaHostAlloc(reinterpret_cast<void **>(&sl.stage), want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        sl.stage = nullptr;
        return TL_ERR_NO_MEMORY;
    }
    sl.stage_bytes = want;
    return TL_OK;
}

}  // namespace

// Called with mu held: take requests from the head of the queue while the
// tick cap and the arena allow, and place the tick's table scratch.
bool tl_server::form_tick(Slot &, std::vector<Req *> &batch, size_t &scratch_off, size_t &scratch_bytes)
{
    const int64_t cap = cfg.max_points_per_tick;
    int64_t pts = 0, nsys = 0;
    size_t table = 0;
    while (!pending.empty() && batch.size() < kMaxJobsPerTick) {
        Req *r = pending.front();
        if (!batch.empty() && (cap == 0 || pts + r->d.count > cap)) break;
        const size_t off = arena.alloc(r->bytes);
        if (off == SIZE_MAX) break;
        r->off = off;
        r->layout(off);
        batch.push_back(r);
        pending.pop_front();
        pts += r->d.count;
        nsys += r->systems();
        table += up(r->table_bytes());
    }
    while (!batch.empty()) {
        scratch_bytes = tick_scratch_bytes(table, nsys);
        scratch_off = arena.alloc(scratch_bytes);
        if (scratch_off != SIZE_MAX) return true;
        Req *r = batch.back();  // give the last request back and retry
        batch.pop_back();
        arena.release(r->off, r->bytes);
        r->off = SIZE_MAX;
        table -= up(r->table_bytes());
        nsys -= r->systems();
        pending.push_front(r);
    }
    return false;
}

// Issue a tick's copies and kernels on the slot's stream (no lock held).
// Each group copies its inputs in, runs, copies its results out and records
// its event, cheapest law class first, so a request waits only for its own
// group and the groups issued before it.
tl_status tl_server::enqueue(Slot &sl, std::vector<Req *> &batch)
{
    cudaStream_t st = sl.stream, s_in = sl.s_in, s_out = sl.s_out;
    cudaError_t e = cudaSuccess;
    auto dptr = [&](size_t off) { return base + off; };
    sl.groups.clear();
    std::map<std::pair<int, int>, std::vector<Req *>> classes;  // (law, n): Norton first, then tanh by n
    std::vector<Req *> solves, empties;
    size_t need = 0, nsys = 0;
    for (Req *r : batch) {
        need += up(r->table_bytes());
        if (r->d.count == 0) empties.push_back(r);
        else if (r->d.kind == TL_REQ_NEWTON) classes[{r->d.law.id, r->d.law.n}].push_back(r);
        else {
            solves.push_back(r);
            nsys += static_cast<size_t>(r->d.count);
        }
    }
    tl_status ts = grow_stage(sl, need + 4 * Arena::kAlign);
    if (ts != TL_OK) return ts;
    auto close_group = [&](std::vector<Req *> &reqs, bool timed) -> tl_status {
        const size_t g = sl.groups.size();
        if (g >= sl.evs.size()) return TL_ERR_UNSUPPORTED;
        const cudaError_t er = cudaEventRecord(sl.evs[g], s_out);
        if (er != cudaSuccess) return fail_cuda(sl.h, er);
        sl.groups.push_back(Group{reqs, false, timed});
        return TL_OK;
    };
    // the group's inputs are on the device: its kernels may start
    auto inputs_ready = [&](size_t g) -> cudaError_t {
        cudaError_t er = cudaEventRecord(sl.ev_in[g], s_in);
        if (er == cudaSuccess) er = cudaStreamWaitEvent(st, sl.ev_in[g], 0);
        return er;
    };
    // the group's kernels are done: its results may go home
    auto kernels_done = [&](size_t g) -> cudaError_t {
        cudaError_t er = cudaEventRecord(sl.ev_k[g], st);
        if (er == cudaSuccess) er = cudaStreamWaitEvent(s_out, sl.ev_k[g], 0);
        return er;
    };
    auto copy_in = [&](Req *r) -> cudaError_t {
        const size_t c = static_cast<size_t>(r->d.count);
        if (r->d.kind == TL_REQ_NEWTON) {
            const size_t ld = r->d.ld_in > 0 ? static_cast<size_t>(r->d.ld_in) : c;
            if (ld == c)
                return cudaMemcpyAsync(dptr(r->o_in), r->d.in, c * r->fields() * 8, cudaMemcpyHostToDevice, s_in);
            return cudaMemcpy2DAsync(dptr(r->o_in), c * 8, r->d.in, ld * 8, c * 8, static_cast<size_t>(r->fields()),
                                     cudaMemcpyHostToDevice, s_in);
        }
        const size_t n = static_cast<size_t>(r->d.n);
        cudaError_t er = cudaMemcpyAsync(dptr(r->o_in), r->d.in, c * n * n * 8, cudaMemcpyHostToDevice, s_in);
        if (er == cudaSuccess) er = cudaMemcpyAsync(dptr(r->o_x), r->d.rhs, c * n * 8, cudaMemcpyHostToDevice, s_in);
        return er;
    };
    auto copy_out = [&](Req *r) -> cudaError_t {
        const size_t c = static_cast<size_t>(r->d.count);
        cudaError_t er;
        if (r->d.kind == TL_REQ_NEWTON) {
            er = cudaMemcpyAsync(r->d.x, dptr(r->o_x), c * r->xrows() * 8, cudaMemcpyDeviceToHost, s_out);
            if (er == cudaSuccess && r->has_aux())
                er = cudaMemcpyAsync(r->d.aux, dptr(r->o_aux), c * 6 * 8, cudaMemcpyDeviceToHost, s_out);
            if (er == cudaSuccess) er = cudaMemcpyAsync(r->d.i1, dptr(r->o_i1), c * 4, cudaMemcpyDeviceToHost, s_out);
            if (er == cudaSuccess) er = cudaMemcpyAsync(r->d.i2, dptr(r->o_i2), c * 4, cudaMemcpyDeviceToHost, s_out);
        } else {
            const size_t n = static_cast<size_t>(r->d.n);
            er = cudaMemcpyAsync(r->d.x, dptr(r->o_x), c * n * 8, cudaMemcpyDeviceToHost, s_out);
            if (er == cudaSuccess)
                er = cudaMemcpyAsync(r->d.i1, dptr(r->o_i1), c * n * 4, cudaMemcpyDeviceToHost, s_out);
        }
        return er;
    };

    if (!empties.empty() && (ts = close_group(empties, false)) != TL_OK) return ts;
    size_t cur = 0;  // offset inside both the staging buffer and the scratch block
    for (auto &kv : classes) {
        for (Req *r : kv.second)
            if ((e = copy_in(r)) != cudaSuccess) return fail_cuda(sl.h, e);
        const size_t tb = up(kv.second.size() * sizeof(NewtonJob));
        NewtonJob *jobs = reinterpret_cast<NewtonJob *>(sl.stage + cur);
        int64_t start = 0;
        for (size_t j = 0; j < kv.second.size(); ++j) {
            Req *r = kv.second[j];
            NewtonJob jb = r->job;
            jb.in = reinterpret_cast<const double *>(dptr(r->o_in));
            jb.x = reinterpret_cast<double *>(dptr(r->o_x));
            jb.out = r->has_aux() ? reinterpret_cast<double *>(dptr(r->o_aux)) : nullptr;
            jb.tangent = nullptr;
            jb.iters = reinterpret_cast<int32_t *>(dptr(r->o_i1));
            jb.status = reinterpret_cast<int32_t *>(dptr(r->o_i2));
            jb.npoints = r->d.count;
            jb.start = start;
            start += r->d.count;
            jobs[j] = jb;
        }
        char *dtab = dptr(sl.scratch_off + cur);
        e = cudaMemcpyAsync(dtab, jobs, kv.second.size() * sizeof(NewtonJob), cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = inputs_ready(sl.groups.size());
        if (e != cudaSuccess) return fail_cuda(sl.h, e);
        NewtonBatch B{};
        B.jobs = reinterpret_cast<const NewtonJob *>(dtab);
        B.njobs = static_cast<int>(kv.second.size());
        B.total = start;
        B.rtol = cfg.rtol;
        B.max_iter = cfg.max_iter;
        const size_t g = sl.groups.size();
        if (g >= sl.evs.size()) return TL_ERR_UNSUPPORTED;
        cudaEventRecord(sl.kev[2 * g], st);
        ts = newton_launch(sl.h, kv.first.first, kv.first.second, B, st);
        if (ts != TL_OK) return ts;
        cudaEventRecord(sl.kev[2 * g + 1], st);
        if ((e = kernels_done(g)) != cudaSuccess) return fail_cuda(sl.h, e);
        cur += tb;
        for (Req *r : kv.second)
            if ((e = copy_out(r)) != cudaSuccess) return fail_cuda(sl.h, e);
        if ((ts = close_group(kv.second, true)) != TL_OK) return ts;
    }
    if (nsys > 0) {
        for (Req *r : solves)
            if ((e = copy_in(r)) != cudaSuccess) return fail_cuda(sl.h, e);
        // n (int32), a_off, b_off, piv_off (int64), info (int32): element
        // offsets relative to the arena base
        int32_t *hn = reinterpret_cast<int32_t *>(sl.stage + cur);
        int64_t *ha = reinterpret_cast<int64_t *>(sl.stage + cur + up(nsys * 4));
        int64_t *hb = ha + nsys;
        int64_t *hp = hb + nsys;
        const size_t o_n = cur, o_a = cur + up(nsys * 4), o_info = o_a + up(nsys * 24);
        const size_t o_ws = o_info + up(nsys * 4);
        size_t q = 0;
        for (Req *r : solves) {
            const int64_t n = r->d.n;
            for (int64_t s = 0; s < r->d.count; ++s, ++q) {
                hn[q] = static_cast<int32_t>(n);
                ha[q] = static_cast<int64_t>(r->o_in / 8) + s * n * n;
                hb[q] = static_cast<int64_t>(r->o_x / 8) + s * n;
                hp[q] = static_cast<int64_t>(r->o_i1 / 4) + s * n;
            }
        }
        e = cudaMemcpyAsync(dptr(sl.scratch_off + o_n), hn, o_info - o_n, cudaMemcpyHostToDevice, s_in);
        if (e == cudaSuccess) e = inputs_ready(sl.groups.size());
        if (e != cudaSuccess) return fail_cuda(sl.h, e);
        const int32_t *dn = reinterpret_cast<const int32_t *>(dptr(sl.scratch_off + o_n));
        const int64_t *da = reinterpret_cast<const int64_t *>(dptr(sl.scratch_off + o_a));
        int32_t *dinfo = reinterpret_cast<int32_t *>(dptr(sl.scratch_off + o_info));
        const double *dbase = reinterpret_cast<const double *>(base);
        // the ragged solve of tl_lupp_solve_batched (binary64) with its bucket
        // workspace in this tick's scratch block
        RaggedArgs ra{nullptr, nullptr, da, dbase, da + nsys, dbase, reinterpret_cast<double *>(base),
                      da + 2 * nsys, reinterpret_cast<int32_t *>(base), dinfo};
        int32_t *dws = reinterpret_cast<int32_t *>(dptr(sl.scratch_off + o_ws));
        const size_t g = sl.groups.size();
        if (g >= sl.evs.size()) return TL_ERR_UNSUPPORTED;
        cudaEventRecord(sl.kev[2 * g], st);
        ts = ragged_solve(sl.h, static_cast<int64_t>(nsys), dn, ra, dws, st);
        if (ts != TL_OK) return ts;
        cudaEventRecord(sl.kev[2 * g + 1], st);
        if ((e = kernels_done(g)) != cudaSuccess) return fail_cuda(sl.h, e);
        q = 0;
        for (Req *r : solves) {
            const size_t c = static_cast<size_t>(r->d.count);
            e = cudaMemcpyAsync(r->d.i2, dinfo + q, c * 4, cudaMemcpyDeviceToHost, s_out);
            if (e == cudaSuccess) e = copy_out(r);
            if (e != cudaSuccess) return fail_cuda(sl.h, e);
            q += c;
        }
        if ((ts = close_group(solves, true)) != TL_OK) return ts;
    }
    return TL_OK;
}

// Called with mu held: one group of a tick ended with `status`.
void tl_server::finish_group(Slot &sl, Group &g, int32_t status)
{
    const size_t gi = static_cast<size_t>(&g - sl.groups.data());
    if (status == TL_OK && gi < sl.groups.size() && 2 * gi + 1 < sl.kev.size() && g.timed) {
        float a = 0.f, b = 0.f;
        if (cudaEventElapsedTime(&a, t0_ev, sl.kev[2 * gi]) == cudaSuccess &&
            cudaEventElapsedTime(&b, t0_ev, sl.kev[2 * gi + 1]) == cudaSuccess && b >= a)
            kernel_spans.emplace_back(a, b);
        cudaGetLastError();
    }
    const Clock::time_point now = Clock::now();
    for (Req *r : g.reqs) {
        r->done = true;
        r->status = status;
        r->t_done = now;
        if (r->off != SIZE_MAX) arena.release(r->off, r->bytes);
        r->off = SIZE_MAX;
        if (status == TL_OK) {
            ++stats.completed;
            stats.points += r->d.count;
        } else {
            ++stats.failed;
        }
    }
    g.done = true;
    cv_done.notify_all();
}

// Called with mu held: finish the groups whose events completed (all of
// them, with `failed` for the requests no group recorded, when failed is
// not TL_OK and the stream has drained); free the slot when none is left.
void tl_server::retire(Slot &sl, tl_status failed)
{
    for (size_t g = 0; g < sl.groups.size(); ++g) {
        Group &gr = sl.groups[g];
        if (gr.done) continue;
        const cudaError_t q = cudaEventQuery(sl.evs[g]);
        if (q == cudaErrorNotReady) return;  // later groups are behind it on the stream
        if (q != cudaSuccess) {
            cudaGetLastError();
            h->last_cuda_error = static_cast<int>(q);
        }
        finish_group(sl, gr, q == cudaSuccess ? TL_OK : TL_ERR_CUDA);
    }
    if (failed != TL_OK) {
        Group rest;
        for (Req *r : sl.reqs)
            if (!r->done) rest.reqs.push_back(r);
        if (!rest.reqs.empty()) finish_group(sl, rest, failed);
    }
    if (sl.scratch_off != SIZE_MAX) arena.release(sl.scratch_off, sl.scratch_bytes);
    sl.scratch_off = SIZE_MAX;
    sl.reqs.clear();
    sl.groups.clear();
    sl.busy = false;
}

void tl_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // retire finished ticks
        bool any_busy = false;
        for (Slot &sl : slots) {
            if (!sl.busy) continue;
            retire(sl, TL_OK);
            if (sl.busy) any_busy = true;
        }
        if (stop && pending.empty() && !any_busy) break;
        // admit the head of the queue into a free slot
        Slot *free_slot = nullptr;
        for (Slot &sl : slots)
            if (!sl.busy) {
                free_slot = &sl;
                break;
            }
        bool launched = false;
        if (free_slot && !pending.empty() && !paused) {
            const Clock::time_point t_host = Clock::now();
            std::vector<Req *> batch;
            size_t soff = SIZE_MAX, sbytes = 0;
            if (form_tick(*free_slot, batch, soff, sbytes)) {
                Slot &sl = *free_slot;
                sl.busy = true;
                sl.reqs = batch;
                sl.scratch_off = soff;
                sl.scratch_bytes = sbytes;
                ++stats.ticks;
                if (stats.arena_high_water < arena.high_water()) stats.arena_high_water = arena.high_water();
                lk.unlock();
                const tl_status ts = enqueue(sl, batch);
                lk.lock();
                stats.host_enqueue_s += std::chrono::duration<double>(Clock::now() - t_host).count();
                if (ts != TL_OK) {
                    // whatever was issued drains before the slot is reused
                    cudaStreamSynchronize(sl.s_in);
                    cudaStreamSynchronize(sl.stream);
                    cudaStreamSynchronize(sl.s_out);
                    cudaGetLastError();
                    retire(sl, ts);
                }
                launched = true;
            } else if (!any_busy) {
                // nothing runs and the head still does not fit: it never will
                Req *r = pending.front();
                pending.pop_front();
                r->done = true;
                r->status = TL_ERR_NO_MEMORY;
                r->t_done = Clock::now();
                ++stats.failed;
                cv_done.notify_all();
                launched = true;
            }
        }
        if (launched) continue;
        if (any_busy) cv_work.wait_for(lk, std::chrono::microseconds(20));
        else cv_work.wait(lk, [&] { return stop || (!pending.empty() && !paused); });
    }
}

extern "C" tl_status tl_server_create(tl_handle *h, const tl_server_config *cfg, tl_server **out)
{
    if (!h) return TL_ERR_INVALID_ARG;
    if (!cfg || !out) return fail_arg(h, cfg ? 3 : 2);
    if (cfg->budget_bytes < (1u << 20) || cfg->slots < 1 || cfg->slots > kMaxSlots || cfg->max_points_per_tick < 0 ||
        !(cfg->rtol >= 0.0) || cfg->max_iter < 0)
        return fail_arg(h, 2);
    *out = nullptr;
    tl_server *s = new tl_server();
    s->h = h;
    s->device = h->device;
    s->cfg = *cfg;
    cudaError_t e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s->base), cfg->budget_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return TL_ERR_NO_MEMORY;
    }
    s->arena.reset(cfg->budget_bytes);
    s->slots.resize(static_cast<size_t>(cfg->slots));
    bool t0_ok = cudaEventCreate(&s->t0_ev) == cudaSuccess && cudaEventRecord(s->t0_ev, nullptr) == cudaSuccess &&
                 cudaEventSynchronize(s->t0_ev) == cudaSuccess;
    if (!t0_ok) {
        cudaGetLastError();
        tl_server_destroy(s);
        return TL_ERR_CUDA;
    }
    for (Slot &sl : s->slots) {
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&sl.s_in, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&sl.s_out, cudaStreamNonBlocking) == cudaSuccess && tl_create(&sl.h) == TL_OK;
        for (std::vector<cudaEvent_t> *v : {&sl.evs, &sl.ev_in, &sl.ev_k}) {
            for (int g = 0; ok && g < kMaxGroups; ++g) {
                cudaEvent_t ev = nullptr;
                ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
                if (ok) v->push_back(ev);
            }
        }
        for (int g = 0; ok && g < 2 * kMaxGroups; ++g) {
            cudaEvent_t ev = nullptr;
            ok = cudaEventCreate(&ev) == cudaSuccess;
            if (ok) sl.kev.push_back(ev);
        }
        if (!ok) {
            cudaGetLastError();
            tl_server_destroy(s);
            return TL_ERR_CUDA;
        }
    }
    s->loop = std::thread([s] { s->run(); });
    *out = s;
    return TL_OK;
}

extern "C" tl_status tl_server_submit(tl_server *s, const tl_request *req, int64_t *id)
{
    if (!s || !id) return TL_ERR_INVALID_ARG;
    const tl_status st = check_request(req);
    if (st != TL_OK) return st;
    Req *r = new Req();
    r->d = *req;
    if (req->kind == TL_REQ_NEWTON) law_params(req->law, &r->job);
    r->bytes = r->layout(0);
    if (r->bytes + tick_scratch_bytes(up(r->table_bytes()), r->systems()) > s->arena.capacity()) {
        delete r;
        return TL_ERR_NO_MEMORY;
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return TL_ERR_INVALID_ARG;
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        ++s->stats.submitted;
        s->pending.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_one();
    return TL_OK;
}

namespace {

tl_status report(tl_server *s, std::unordered_map<int64_t, Req *>::iterator it, int32_t *req_status, double *latency_s)
{
    Req *r = it->second;
    if (req_status) *req_status = r->status;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    s->reqs.erase(it);
    delete r;
    return TL_OK;
}

}  // namespace

extern "C" tl_status tl_server_test(tl_server *s, int64_t id, int32_t *done, int32_t *req_status, double *latency_s)
{
    if (!s || !done) return TL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return TL_ERR_INVALID_ARG;
    *done = it->second->done ? 1 : 0;
    if (!*done) return TL_OK;
    return report(s, it, req_status, latency_s);
}

extern "C" tl_status tl_server_wait(tl_server *s, int64_t id, double timeout_s, int32_t *req_status, double *latency_s)
{
    if (!s || !(timeout_s >= 0.0)) return TL_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return TL_ERR_INVALID_ARG;
    Req *r = it->second;
    const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    if (!s->cv_done.wait_until(lk, limit, [&] { return r->done; })) return TL_ERR_TIMEOUT;
    return report(s, s->reqs.find(id), req_status, latency_s);
}

// Called with mu held: the union of the recorded kernel intervals (the time
// at least one of the server's kernels ran), in seconds.
double tl_server::busy_union()
{
    if (kernel_spans.empty()) return 0.0;
    std::sort(kernel_spans.begin(), kernel_spans.end());
    double busy = 0.0;
    float a = kernel_spans[0].first, b = kernel_spans[0].second;
    for (size_t i = 1; i < kernel_spans.size(); ++i) {
        if (kernel_spans[i].first > b) {
            busy += b - a;
            a = kernel_spans[i].first;
        }
        b = std::max(b, kernel_spans[i].second);
    }
    return (busy + (b - a)) * 1e-3;
}

extern "C" tl_status tl_server_pause(tl_server *s, int paused)
{
    if (!s) return TL_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv_work.notify_all();
    return TL_OK;
}

extern "C" tl_status tl_server_stats_get(tl_server *s, tl_server_stats *out)
{
    if (!s || !out) return TL_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->kernel_busy_s = s->busy_union();
    out->arena_high_water = s->arena.high_water();
    return TL_OK;
}

extern "C" tl_status tl_server_destroy(tl_server *s)
{
    if (!s) return TL_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->paused = false;  // queued requests still finish
    }
    s->cv_work.notify_all();
    if (s->loop.joinable()) s->loop.join();
    for (Slot &sl : s->slots) {
        for (cudaStream_t x : {sl.s_in, sl.stream, sl.s_out})
            if (x) cudaStreamSynchronize(x);
        for (std::vector<cudaEvent_t> *v : {&sl.evs, &sl.ev_in, &sl.ev_k, &sl.kev})
            for (cudaEvent_t ev : *v) cudaEventDestroy(ev);
        for (cudaStream_t x : {sl.s_in, sl.stream, sl.s_out})
            if (x) cudaStreamDestroy(x);
        if (sl.h) tl_destroy(sl.h);
        if (sl.stage) cudaFreeHost(sl.stage);
    }
    cudaFree(s->base);
    if (s->t0_ev) cudaEventDestroy(s->t0_ev);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return TL_OK;
}
