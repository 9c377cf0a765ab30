// Scan server: continuous batching of COUNT/SUM queries against a device-
// resident table of columns.
//
// A query names 1..k table columns, each with its own range predicate.  The
// server admits a query when its entries fit the device-memory budget of an
// in-flight batch; a dispatcher thread packs every admitted query it finds
// into one batched launch (the persistent batch kernel) on a free slot's
// stream, so batches that arrive while others run overlap on the device; a
// completion thread waits for the oldest in-flight batch, hands each query
// its results and frees the slot, which lets the dispatcher admit more.
// Results are bit-identical to a query run alone: each entry is an
// independent exact scan.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gbscan.h"
#include "batch_kernels.cuh"

void gb_set_last_error(const char* msg);
bool gb_column_view(const scan_column* c, const uint32_t** packed, uint64_t* n, uint32_t* b,
                    uint32_t* base, const uint2** zonemap);

namespace {

using Clock = std::chrono::steady_clock;

scan_status sfail(scan_status s, const char* msg)
{
    gb_set_last_error(msg);
    return s;
}

struct Query {
    uint64_t id = 0;
    std::vector<uint32_t> cols;
    std::vector<scan_pred> preds;
    std::vector<scan_result> results;
    Clock::time_point arrived, done_at;
    bool done = false;
};

constexpr size_t kCtlWords = 40;  // per slot: one pop counter per width (u32), status at u32 index 33

struct Group {
    uint32_t b, first, count, ntiles;
};

struct Slot {
    std::vector<Group> groups;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    gb::BatchCol* h_tab = nullptr;
    gb::BatchCol* d_tab = nullptr;
    unsigned long long* d_res = nullptr;  // 4 words per entry + control
    unsigned long long* h_res = nullptr;
    uint32_t cap = 0;
    std::vector<Query*> queries;
    uint32_t entries = 0;
    bool busy = false;
};

}  // namespace

struct scan_server {
    std::vector<const scan_column*> table;
    std::vector<uint32_t> width;  // b of every table column
    std::vector<Slot> slots;
    uint32_t max_entries_per_batch = 0;
    uint32_t max_queue = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Query*> pending;
    std::deque<int> inflight;  // slot indices in launch order
    std::unordered_map<uint64_t, Query*> queries;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread dispatcher, completer;
    int sms = 1;
    // statistics
    uint64_t batches = 0, entries_launched = 0, rejected = 0;
    std::atomic<unsigned int> device_error{0};
    char error_text[256] = {0};  // first device-side failure, under mu
};

namespace {

uint32_t tile_blocks_for(uint32_t b) { return gb::batch_tile_blocks(b); }

void fill_entry(gb::BatchCol& d, const scan_column* col, scan_pred pr, uint32_t out, uint32_t& tiles)
// tiles: running tile count of the entry's width group (numbering restarts per group)
{
    const uint2* zm = nullptr;
    const uint32_t* pk;
    uint64_t n;
    uint32_t b, base;
    gb_column_view(col, &pk, &n, &b, &base, &zm);
    std::memset(&d, 0, sizeof d);
    d.packed = pk;
    d.zonemap = zm;
    d.n = n;
    d.b = b;
    d.base = base;
    d.tile_blocks = tile_blocks_for(b);
    d.tile_begin = tiles;
    d.out = out;
    const int64_t lo_v = static_cast<int64_t>(base), hi_v = lo_v + (1ll << b);
    const int64_t lo = std::max(pr.lo, lo_v), hi = std::min(pr.hi, hi_v);
    d.flags = zm ? gb::kColZone : 0u;  // zone maps are exact: skip wherever one exists
    if (lo >= hi || n == 0) {
        d.flags |= gb::kColEmpty;
    } else {
        d.lo = static_cast<uint32_t>(lo - lo_v);
        d.wm1 = static_cast<uint32_t>(hi - lo - 1);
        d.zlo = static_cast<uint64_t>(lo);
        d.zhi = static_cast<uint64_t>(hi);
    }
    const uint64_t nblocks = (n + 1023u) >> 10;
    tiles += static_cast<uint32_t>((nblocks + d.tile_blocks - 1) / d.tile_blocks);
}

// Launch one slot's batch (descriptors in h_tab, grouped by width); *step names a failing call.
cudaError_t launch_slot(scan_server* sv, Slot& s, const char** step)
{
    const uint32_t n = s.entries;
    *step = "descriptor copy";
    cudaError_t e = cudaMemcpyAsync(s.d_tab, s.h_tab, n * sizeof(gb::BatchCol), cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) {
        *step = "result reset";
        e = cudaMemsetAsync(s.d_res, 0, (4ull * s.cap + kCtlWords) * sizeof(unsigned long long), s.stream);
    }
    unsigned int* ctl = reinterpret_cast<unsigned int*>(s.d_res + 4ull * s.cap);
    const uint32_t warps = static_cast<uint32_t>(sv->sms) * gb::kBatchWarps;
    for (size_t gi = 0; e == cudaSuccess && gi < s.groups.size(); ++gi) {
        const Group& g = s.groups[gi];
        if (!g.ntiles) continue;
        *step = "batch kernel launch";
        gb::BatchParams p{};
        p.cols = s.d_tab + g.first;
        p.ncols = g.count;
        p.ntiles = g.ntiles;
        p.chunk = std::max<uint32_t>(1, std::min<uint32_t>(256, g.ntiles / (8 * warps)));
        p.head = ctl + gi;
        p.results = s.d_res;
        p.status = ctl + 33;
        // the default batch shape (the tiles were cut by batch_tile_blocks) and
        // two CTAs per SM, which that shape fits: the kernels of concurrent
        // slots then share every SM.  One CTA per SM kept half the bytes in
        // flight: at 0.9x the serial capacity p50 was 400 us against 295 us,
        // and at 1.5x the queue grew (p50 37 ms) where it now serves every
        // query (p50 0.55 ms).
        p.stages = gb::kBatchStages;
        p.slot_bytes = gb::batch_tile_blocks(g.b) * 128u * g.b;
        e = gb_launch_batch(false, static_cast<int>(g.b), p, gb::batch_default_warps(g.b), 2 * sv->sms, s.stream);
    }
    if (e == cudaSuccess) {
        // results of the n entries, then the control words (pop counters, status)
        *step = "result copy";
        e = cudaMemcpyAsync(s.h_res, s.d_res, 4ull * n * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.h_res + 4ull * s.cap, s.d_res + 4ull * s.cap, kCtlWords * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, s.stream);
    }
    if (e == cudaSuccess) {
        *step = "completion event";
        e = cudaEventRecord(s.done, s.stream);
    }
    return e;
}

void note_error(scan_server* sv, const char* step, cudaError_t e)
{
    if (!sv->error_text[0])
        snprintf(sv->error_text, sizeof sv->error_text, "%s: %s", step,
                 e == cudaSuccess ? "device wait timed out" : cudaGetErrorString(e));
}

void dispatcher_loop(scan_server* sv)
{
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        int free_slot = -1;
        sv->cv_work.wait(lk, [&] {
            if (sv->stop) return true;
            if (sv->pending.empty()) return false;
            for (size_t i = 0; i < sv->slots.size(); ++i)
                if (!sv->slots[i].busy) {
                    free_slot = static_cast<int>(i);
                    return true;
                }
            return false;
        });
        if (sv->stop) return;
        Slot& s = sv->slots[free_slot];
        // admit every pending query that fits this slot's memory
        s.queries.clear();
        s.entries = 0;
        uint32_t tiles = 0;
        std::vector<std::pair<uint32_t, uint32_t>> scans;  // (width, entry) of every column scan
        while (!sv->pending.empty()) {
            Query* q = sv->pending.front();
            if (s.entries + q->cols.size() > s.cap) break;
            sv->pending.pop_front();
            for (size_t j = 0; j < q->cols.size(); ++j)
                scans.emplace_back(sv->width[q->cols[j]], static_cast<uint32_t>(s.entries + j));
            s.entries += static_cast<uint32_t>(q->cols.size());
            s.queries.push_back(q);
        }
        // descriptor order by width (instruction-cache locality); results stay per entry
        std::stable_sort(scans.begin(), scans.end());
        std::vector<std::pair<uint32_t, scan_pred>> entry_src(s.entries);
        {
            uint32_t e = 0;
            for (Query* q : s.queries)
                for (size_t j = 0; j < q->cols.size(); ++j, ++e) entry_src[e] = {q->cols[j], q->preds[j]};
        }
        s.groups.clear();
        for (uint32_t pos = 0; pos < scans.size(); ++pos) {
            const uint32_t e = scans[pos].second;
            if (s.groups.empty() || s.groups.back().b != scans[pos].first) {
                s.groups.push_back({scans[pos].first, pos, 0, 0});
                tiles = 0;
            }
            fill_entry(s.h_tab[pos], sv->table[entry_src[e].first], entry_src[e].second, e, tiles);
            s.groups.back().count += 1;
            s.groups.back().ntiles = tiles;
        }
        if (s.queries.empty()) continue;  // cannot happen: queries are capped at submit
        s.busy = true;  // reserved: the dispatcher alone touches it until it is published
        sv->batches += 1;
        sv->entries_launched += s.entries;
        lk.unlock();
        const char* step = "";
        const cudaError_t e = launch_slot(sv, s, &step);
        lk.lock();
        if (e != cudaSuccess) {
            sv->device_error.fetch_or(1u);
            note_error(sv, step, e);
        }
        // publish only now: the completion event of this batch has been recorded
        sv->inflight.push_back(free_slot);
        sv->cv_done.notify_all();
    }
}

void completer_loop(scan_server* sv)
{
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        sv->cv_done.wait(lk, [&] { return sv->stop || !sv->inflight.empty(); });
        if (sv->inflight.empty() && sv->stop) return;
        const int si = sv->inflight.front();
        Slot& s = sv->slots[si];
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(s.done);
        const auto now = Clock::now();
        lk.lock();
        if (e != cudaSuccess) {
            sv->device_error.fetch_or(1u);
            note_error(sv, "completion wait", e);
        }
        const unsigned int status = reinterpret_cast<const unsigned int*>(s.h_res + 4ull * s.cap)[33];
        if (status) {
            sv->device_error.fetch_or(2u);
            note_error(sv, "batch kernel", cudaSuccess);
        }
        uint32_t k = 0;
        for (Query* q : s.queries) {
            q->results.resize(q->cols.size());
            for (size_t j = 0; j < q->cols.size(); ++j, ++k)
                std::memcpy(&q->results[j], s.h_res + 4ull * k, sizeof(scan_result));
            q->done_at = now;
            q->done = true;
        }
        s.queries.clear();
        s.busy = false;
        sv->inflight.pop_front();
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

scan_status scan_server_create(scan_column* const* cols, uint32_t ncols, uint32_t slots,
                               uint64_t device_bytes_per_slot, uint32_t max_queue, scan_server** out)
{
    gb_set_last_error("");
    if (!out || !cols || !ncols || !slots || slots > 16) return sfail(SCAN_EINVAL, "bad server arguments");
    *out = nullptr;
    const uint64_t per_entry = sizeof(gb::BatchCol) + 4 * sizeof(unsigned long long);
    const uint64_t cap = device_bytes_per_slot / per_entry;
    if (cap < 8) return sfail(SCAN_EINVAL, "device_bytes_per_slot admits fewer than 8 column scans");
    auto* sv = new (std::nothrow) scan_server();
    if (!sv) return sfail(SCAN_ENOMEM, "host allocation failed");
    sv->table.assign(cols, cols + ncols);
    for (uint32_t i = 0; i < ncols; ++i) {
        const uint2* zm = nullptr;
        const uint32_t* pk;
        uint64_t n;
        uint32_t b = 0, base;
        if (!cols[i] || !gb_column_view(cols[i], &pk, &n, &b, &base, &zm)) {
            delete sv;
            return sfail(SCAN_EINVAL, "a table column is NULL or not lane-interleaved");
        }
        sv->width.push_back(b);
    }
    sv->max_entries_per_batch = static_cast<uint32_t>(std::min<uint64_t>(cap, 1u << 20));
    sv->max_queue = max_queue ? max_queue : 4096;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, dev);
    sv->slots.resize(slots);
    for (auto& s : sv->slots) {
        s.cap = sv->max_entries_per_batch;
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&s.h_tab), s.cap * sizeof(gb::BatchCol));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.d_tab), s.cap * sizeof(gb::BatchCol));
        if (e == cudaSuccess)
            e = cudaMalloc(reinterpret_cast<void**>(&s.d_res), (4ull * s.cap + kCtlWords) * sizeof(unsigned long long));
        if (e == cudaSuccess)
            e = cudaMallocHost(reinterpret_cast<void**>(&s.h_res), (4ull * s.cap + kCtlWords) * sizeof(unsigned long long));
        if (e != cudaSuccess) {
            scan_server_destroy(sv);
            return sfail(e == cudaErrorMemoryAllocation ? SCAN_ENOMEM : SCAN_ECUDA, "server slot allocation");
        }
    }
    sv->dispatcher = std::thread(dispatcher_loop, sv);
    sv->completer = std::thread(completer_loop, sv);
    *out = sv;
    return SCAN_OK;
}

scan_status scan_server_submit(scan_server* sv, const uint32_t* col_ids, const scan_pred* preds, uint32_t n,
                               uint64_t* query_id)
{
    gb_set_last_error("");
    if (!sv || !col_ids || !preds || !query_id || !n) return sfail(SCAN_EINVAL, "bad query");
    if (n > sv->max_entries_per_batch) return sfail(SCAN_EINVAL, "query larger than one batch slot");
    for (uint32_t j = 0; j < n; ++j)
        if (col_ids[j] >= sv->table.size()) return sfail(SCAN_EINVAL, "column id out of range");
    auto* q = new (std::nothrow) Query();
    if (!q) return sfail(SCAN_ENOMEM, "host allocation failed");
    q->cols.assign(col_ids, col_ids + n);
    q->preds.assign(preds, preds + n);
    q->arrived = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->pending.size() >= sv->max_queue) {
        sv->rejected += 1;
        delete q;
        return sfail(SCAN_EBUSY, "admission queue is full");
    }
    q->id = sv->next_id++;
    sv->queries[q->id] = q;
    sv->pending.push_back(q);
    *query_id = q->id;
    sv->cv_work.notify_all();
    return SCAN_OK;
}

scan_status scan_server_submit_many(scan_server* sv, uint32_t nqueries, const uint32_t* offsets,
                                    const uint32_t* col_ids, const scan_pred* preds, uint64_t* query_ids)
{
    gb_set_last_error("");
    if (!sv || !offsets || !col_ids || !preds || !query_ids) return sfail(SCAN_EINVAL, "null pointer");
    std::vector<Query*> made;
    made.reserve(nqueries);
    const auto now = Clock::now();
    for (uint32_t k = 0; k < nqueries; ++k) {
        const uint32_t a = offsets[k], b = offsets[k + 1];
        if (b <= a || b - a > sv->max_entries_per_batch) {
            for (Query* q : made) delete q;
            return sfail(SCAN_EINVAL, "a query is empty or larger than one batch slot");
        }
        for (uint32_t j = a; j < b; ++j)
            if (col_ids[j] >= sv->table.size()) {
                for (Query* q : made) delete q;
                return sfail(SCAN_EINVAL, "column id out of range");
            }
        auto* q = new (std::nothrow) Query();
        if (!q) {
            for (Query* x : made) delete x;
            return sfail(SCAN_ENOMEM, "host allocation failed");
        }
        q->cols.assign(col_ids + a, col_ids + b);
        q->preds.assign(preds + a, preds + b);
        q->arrived = now;
        made.push_back(q);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->pending.size() + made.size() > sv->max_queue) {
        sv->rejected += made.size();
        for (Query* q : made) delete q;
        return sfail(SCAN_EBUSY, "admission queue is full");
    }
    for (uint32_t k = 0; k < made.size(); ++k) {
        made[k]->id = sv->next_id++;
        sv->queries[made[k]->id] = made[k];
        sv->pending.push_back(made[k]);
        query_ids[k] = made[k]->id;
    }
    sv->cv_work.notify_all();
    return SCAN_OK;
}

scan_status scan_server_poll(scan_server* sv, uint64_t query_id, int wait, scan_result* out, uint32_t n,
                             double* latency_us, int* done)
{
    gb_set_last_error("");
    if (!sv || !done) return sfail(SCAN_EINVAL, "null pointer");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->queries.find(query_id);
    if (it == sv->queries.end()) return sfail(SCAN_EINVAL, "unknown or already collected query id");
    Query* q = it->second;
    if (wait)
        sv->cv_done.wait(lk, [&] { return q->done || sv->device_error.load() != 0; });
    if (sv->device_error.load()) {
        static thread_local char msg[320];
        snprintf(msg, sizeof msg, "a batch failed on the device (%s)", sv->error_text);
        return sfail((sv->device_error.load() & 2u) ? SCAN_ETIMEOUT : SCAN_ECUDA, msg);
    }
    *done = q->done ? 1 : 0;
    if (!q->done) return SCAN_OK;
    if (n < q->cols.size() || !out) return sfail(SCAN_EINVAL, "result buffer too small");
    std::memcpy(out, q->results.data(), q->results.size() * sizeof(scan_result));
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(q->done_at - q->arrived).count();
    sv->queries.erase(it);
    delete q;
    return SCAN_OK;
}

scan_status scan_server_stats(scan_server* sv, uint64_t* batches, uint64_t* entries, uint64_t* rejected,
                              uint32_t* queued)
{
    if (!sv) return sfail(SCAN_EINVAL, "null pointer");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (batches) *batches = sv->batches;
    if (entries) *entries = sv->entries_launched;
    if (rejected) *rejected = sv->rejected;
    if (queued) *queued = static_cast<uint32_t>(sv->pending.size());
    return SCAN_OK;
}

scan_status scan_server_destroy(scan_server* sv)
{
    if (!sv) return SCAN_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
    if (sv->dispatcher.joinable()) sv->dispatcher.join();
    // let batches still on the GPU finish before their memory goes away
    for (auto& s : sv->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    if (sv->completer.joinable()) sv->completer.join();
    for (auto& s : sv->slots) {
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.h_tab) cudaFreeHost(s.h_tab);
        if (s.h_res) cudaFreeHost(s.h_res);
        if (s.d_tab) cudaFree(s.d_tab);
        if (s.d_res) cudaFree(s.d_res);
    }
    for (auto& kv : sv->queries) delete kv.second;
    for (Query* q : sv->pending) (void)q;  // owned through sv->queries
    delete sv;
    return SCAN_OK;
}

}  // extern "C"
