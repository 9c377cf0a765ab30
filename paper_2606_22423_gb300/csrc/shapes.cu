// Launch shapes of the persistent scan kernels and their autotuner.
//
// Every single-column scan runs one CTA per SM whose warps each stream tiles
// through a ring of shared-memory slots (paper §3's fused decode -> filter ->
// aggregate, with the GPU's copy engine in front of it).  How many warps share
// an SM, how deep the ring is and how many 1024-value blocks make a tile trade
// latency hiding against per-tile overhead and load balance, and the best
// trade differs with the width b: below the ridge the decode is issue-bound
// and more warps hide its dependent chains; above it the copies bind and
// deeper rings or larger tiles pay.  The branchy kernel adds a choice of vote
// form (one value or one row of a thread's lanes per vote, the row as C++ or
// as one PTX block of one or two rows).  Batched scans run two CTAs per SM
// (one of each graph chain), so their shapes stay within half the SM's shared
// memory.
//
// This unit keeps one shape per (kernel kind, b): the built-in rule until a
// tuned shape is installed.  The tuner times every legal candidate on a
// caller's column and installs the fastest; shapes can be saved to and loaded
// from a versioned text file tied to the device they were tuned on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "batch_kernels.cuh"
#include "scan_kernels.cuh"

namespace {

enum Kind : int { kKFullBF = 0, kKFullBR = 1, kKQueueBF = 2, kKQueueBR = 3, kKBatchBF = 4, kKBatchBR = 5, kKinds = 6 };
const char* const kKindName[kKinds] = {"full_bf", "full_br", "queue_bf", "queue_br", "batch_bf", "batch_br"};

struct Entry {
    bool tuned = false;
    gb::LaunchShape shape{};
    float best_us = 0.f, default_us = 0.f;
};

std::mutex g_mu;
Entry g_table[kKinds][33];

int kind_of_op(int op)
{
    switch (op) {
    case gb::kOpFullBF: return kKFullBF;
    case gb::kOpFullBR: return kKFullBR;
    case gb::kOpQueueBF: return kKQueueBF;
    case gb::kOpQueueBR: return kKQueueBR;
    case gb::kOpBatchBF: return kKBatchBF;
    case gb::kOpBatchBR: return kKBatchBR;
    default: return -1;
    }
}

int kind_of_strategy(scan_strategy s)
{
    switch (s) {
    case SCAN_AUTO:
    case SCAN_BRANCHFREE: return kKFullBF;
    case SCAN_BRANCHY: return kKFullBR;
    case SCAN_ZONE_SKIP_BF:
    case SCAN_ZONE_AGG_BF: return kKQueueBF;
    case SCAN_ZONE_SKIP_BR:
    case SCAN_ZONE_AGG_BR: return kKQueueBR;
    default: return -1;
    }
}

bool is_batch(int kind) { return kind == kKBatchBF || kind == kKBatchBR; }

gb::LaunchShape default_shape(int kind, int b)
{
    if (is_batch(kind))
        return gb::LaunchShape{gb::batch_default_warps(static_cast<uint32_t>(b)), gb::kBatchStages,
                               static_cast<int>(gb::batch_tile_blocks(static_cast<uint32_t>(b))), 0, 0};
    const gb::ShapeInfo si = gb::shape_of(b);
    return gb::LaunchShape{si.warps, si.stages, si.tile_blocks, 0, 0};
}

uint32_t smem_of(int kind, int b, const gb::LaunchShape& s)
{
    const uint32_t w = static_cast<uint32_t>(s.warps), st = static_cast<uint32_t>(s.stages);
    const uint32_t tile = static_cast<uint32_t>(s.tile_blocks) * 128u * static_cast<uint32_t>(b);
    return is_batch(kind) ? gb::batch_smem_bytes(w, st, tile)
                          : gb::pipe_smem_bytes(static_cast<uint32_t>(b), w, st, static_cast<uint32_t>(s.tile_blocks));
}

int step_of(int b, int vec_lanes = 0) { return vec_lanes ? vec_lanes : gb::default_lpt(b); }

// Legality of a shape for (kind, b); `why` names the first violated rule.
bool shape_ok(int kind, int b, const gb::LaunchShape& s, const char** why)
{
    const bool wide = kind == kKFullBF || kind == kKFullBR || is_batch(kind);  // up to 16 warps, 64-block tiles
    if (b < 1 || b > 32) return *why = "b must be in 1..32", false;
    if (s.vec_lanes != 0 && s.vec_lanes != gb::default_lpt(b) &&
        !(s.vec_lanes == 2 && b >= 9 && b <= 16 && (kind == kKFullBF || kind == kKFullBR)))
        return *why = "vec_lanes is 0, the width's default, or 2 for full scans at b = 9..16", false;
    const int step = step_of(b, s.vec_lanes);
    if (s.warps < 1 || s.warps > (wide ? 16 : 8))
        return *why = wide ? "full and batched scans take 1..16 warps per CTA" : "zone-skip scans take 1..8 warps per CTA",
               false;
    if (s.stages < 1 || s.stages > 6) return *why = "stages must be in 1..6", false;
    if (s.tile_blocks < step || s.tile_blocks % step != 0)
        return *why = "tile_blocks must be a positive multiple of the warp step (vec_lanes blocks; by default 4 for "
                      "b <= 16, else 2)",
               false;
    if (s.tile_blocks > (wide ? 64 : 32))
        return *why = wide ? "full and batched scans take at most 64 blocks per tile" : "zone-skip tiles hold at most 32 blocks",
               false;
    if (s.vote_rows < 0 || s.vote_rows > 3) return *why = "vote_rows must be 0, 1, 2 or 3", false;
    if (s.vote_rows && (kind != kKFullBR || b > 21))
        return *why = "the row vote applies to full branchy scans at b <= 21", false;
    if (smem_of(kind, b, s) > static_cast<uint32_t>(gb::kSmemMax))
        return *why = "the slots do not fit 226 KB of shared memory", false;
    return *why = "", true;
}

// The tuner's search space for (kind, b): 8/12/16 warps (full scans; queue
// scans 8), 2..4 stages, tiles of about 2..24 KB in whole warp steps, and for
// full branchy scans at b <= 21 both vote groups; illegal shapes dropped.
// Batched scans: 4/6/8 warps, 2 or 3 stages, tiles of about 4..12 KB, only
// shapes whose slots leave room for a second CTA on the SM (the graph runs
// two chains of width groups side by side).
std::vector<gb::LaunchShape> candidates(int kind, int b)
{
    const bool full = kind == kKFullBF || kind == kKFullBR || is_batch(kind);
    std::vector<int> geos{0};
    if ((kind == kKFullBF || kind == kKFullBR) && b >= 9 && b <= 16) geos.push_back(2);
    std::vector<int> warps = is_batch(kind) ? std::vector<int>{4, 6, 8}
                             : full           ? std::vector<int>{8, 12, 16}
                                              : std::vector<int>{8};
    const std::vector<int> kbs = is_batch(kind) ? std::vector<int>{4, 6, 8, 12}
                                                : std::vector<int>{2, 4, 6, 8, 12, 16, 24};
    const int votes = (kind == kKFullBR && b <= 21) ? 4 : 1;
    const std::vector<int> stages = is_batch(kind) ? std::vector<int>{2, 3} : std::vector<int>{2, 3, 4};
    std::vector<gb::LaunchShape> out;
    for (int geo : geos) {
        const int step = step_of(b, geo);
        std::vector<int> tiles;
        for (int kb : kbs) {
            int tb = (kb * 1024 / (128 * b)) / step * step;
            tb = std::max(tb, step);
            tb = std::min(tb, is_batch(kind) ? 64 : 32);
            if (std::find(tiles.begin(), tiles.end(), tb) == tiles.end()) tiles.push_back(tb);
        }
        for (int v = 0; v < votes; ++v)
            for (int w : (geo == 2 ? std::vector<int>{12, 16} : warps))
                for (int st : stages)
                    for (int tb : tiles) {
                        const gb::LaunchShape s{w, st, tb, v, geo};
                        const char* why = nullptr;
                        if (is_batch(kind) && smem_of(kind, b, s) > gb::kBatchPairSmem) continue;
                        if (shape_ok(kind, b, s, &why)) out.push_back(s);
                    }
    }
    return out;
}

scan_status shapes_fail(scan_status s, const std::string& msg)
{
    gb_set_last_error(msg.c_str());
    return s;
}

gb::LaunchShape from_abi(const scan_shape& s)
{
    return gb::LaunchShape{static_cast<int>(s.warps), static_cast<int>(s.stages), static_cast<int>(s.tile_blocks),
                           static_cast<int>(s.vote_rows), static_cast<int>(s.vec_lanes)};
}

scan_shape to_abi(const gb::LaunchShape& s)
{
    return scan_shape{static_cast<uint32_t>(s.warps), static_cast<uint32_t>(s.stages),
                      static_cast<uint32_t>(s.tile_blocks), static_cast<uint32_t>(s.vote_rows),
                      static_cast<uint32_t>(s.vec_lanes)};
}

// The device a cache file belongs to: its name (blanks replaced) and SM
// count; "none 0" when no device is visible.
std::string device_identity()
{
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "none 0";
    }
    std::string name = prop.name;
    for (char& ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    return name + " " + std::to_string(prop.multiProcessorCount);
}

constexpr const char* kMagic = "gbscan-shapes";
constexpr int kVersion = 3;  // 2: vec_lanes column; 3: batch shapes for two CTAs per SM

}  // namespace

// Shape of (op, b) for a launch: the installed tuned shape, else the rule.
gb::LaunchShape gb_shape_for(int b, int op)
{
    const int kind = kind_of_op(op);
    if (kind >= 0 && b >= 1 && b <= 32) {
        std::lock_guard<std::mutex> lock(g_mu);
        const Entry& e = g_table[kind][b];
        if (e.tuned) return e.shape;
        return default_shape(kind, b);
    }
    return default_shape(kKFullBF, b);
}

// Candidate shapes of (op, b) for the batch tuner.
std::vector<gb::LaunchShape> gb_shape_candidates(int b, int op)
{
    const int kind = kind_of_op(op);
    if (kind < 0 || b < 1 || b > 32) return {};
    return candidates(kind, b);
}

// Install a shape for (op, b) (nullptr: the rule); false if illegal.
bool gb_shape_install(int b, int op, const gb::LaunchShape* shape, float tuned_us, float rule_us)
{
    const int kind = kind_of_op(op);
    if (kind < 0 || b < 1 || b > 32) return false;
    const char* why = nullptr;
    if (shape && !shape_ok(kind, b, *shape, &why)) return false;
    std::lock_guard<std::mutex> lock(g_mu);
    Entry& e = g_table[kind][b];
    if (!shape) {
        e = Entry{};
        return true;
    }
    e.tuned = true;
    e.shape = *shape;
    e.best_us = tuned_us;
    e.default_us = rule_us;
    return true;
}

namespace {
scan_status kind_shape_get(int kind, uint32_t b, scan_shape* out)
{
    if (!out || kind < 0 || b < 1 || b > 32) return shapes_fail(SCAN_EINVAL, "bad width, kernel or NULL out");
    std::lock_guard<std::mutex> lock(g_mu);
    const Entry& e = g_table[kind][b];
    *out = to_abi(e.tuned ? e.shape : default_shape(kind, static_cast<int>(b)));
    return SCAN_OK;
}

scan_status kind_shape_set(int kind, uint32_t b, const scan_shape* shape)
{
    if (kind < 0 || b < 1 || b > 32) return shapes_fail(SCAN_EINVAL, "bad width or kernel");
    std::lock_guard<std::mutex> lock(g_mu);
    Entry& e = g_table[kind][b];
    if (!shape) {  // back to the built-in rule
        e = Entry{};
        return SCAN_OK;
    }
    const gb::LaunchShape s = from_abi(*shape);
    const char* why = nullptr;
    if (!shape_ok(kind, static_cast<int>(b), s, &why)) return shapes_fail(SCAN_EINVAL, why);
    e.tuned = true;
    e.shape = s;
    e.best_us = e.default_us = 0.f;
    return SCAN_OK;
}

scan_status kind_candidates(int kind, uint32_t b, scan_shape* out, uint32_t capacity, uint32_t* count)
{
    if (!count || kind < 0 || b < 1 || b > 32) return shapes_fail(SCAN_EINVAL, "bad width, kernel or NULL count");
    const std::vector<gb::LaunchShape> c = candidates(kind, static_cast<int>(b));
    *count = static_cast<uint32_t>(c.size());
    if (out)
        for (uint32_t i = 0; i < std::min<uint32_t>(capacity, *count); ++i) out[i] = to_abi(c[i]);
    return SCAN_OK;
}
}  // namespace

extern "C" {

scan_status scan_batch_shape_get(uint32_t b, int branchy, scan_shape* out)
{
    gb_set_last_error("");
    return kind_shape_get(branchy ? kKBatchBR : kKBatchBF, b, out);
}

scan_status scan_batch_shape_set(uint32_t b, int branchy, const scan_shape* shape)
{
    gb_set_last_error("");
    return kind_shape_set(branchy ? kKBatchBR : kKBatchBF, b, shape);
}

scan_status scan_batch_shape_candidates(uint32_t b, int branchy, scan_shape* out, uint32_t capacity,
                                        uint32_t* count)
{
    gb_set_last_error("");
    return kind_candidates(branchy ? kKBatchBR : kKBatchBF, b, out, capacity, count);
}

scan_status scan_shape_get(uint32_t b, scan_strategy strategy, scan_shape* out)
{
    gb_set_last_error("");
    return kind_shape_get(kind_of_strategy(strategy), b, out);
}

scan_status scan_shape_set(uint32_t b, scan_strategy strategy, const scan_shape* shape)
{
    gb_set_last_error("");
    return kind_shape_set(kind_of_strategy(strategy), b, shape);
}

scan_status scan_shape_candidates(uint32_t b, scan_strategy strategy, scan_shape* out, uint32_t capacity,
                                  uint32_t* count)
{
    gb_set_last_error("");
    return kind_candidates(kind_of_strategy(strategy), b, out, capacity, count);
}

scan_status scan_autotune_reset(void)
{
    gb_set_last_error("");
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto& row : g_table)
        for (auto& e : row) e = Entry{};
    return SCAN_OK;
}

scan_status scan_autotune_column(scan_column* col, scan_pred pred, scan_strategy strategy, uint32_t reps,
                                 void* stream, scan_tune_result* out)
{
    gb_set_last_error("");
    const int kind = kind_of_strategy(strategy);
    if (!col || !out || kind < 0 || strategy == SCAN_AUTO)
        return shapes_fail(SCAN_EINVAL, "NULL column or result, or a strategy without its own kernel");
    uint64_t n = 0;
    uint32_t b = 0, base = 0;
    const uint32_t* packed = nullptr;
    const uint2* zm = nullptr;
    if (!gb_column_view(col, &packed, &n, &b, &base, &zm)) return shapes_fail(SCAN_EINVAL, "not a column");
    if (n < 1024) return shapes_fail(SCAN_EINVAL, "tune on a column of at least one whole block");
    reps = std::max<uint32_t>(1, std::min<uint32_t>(reps, 100));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<gb::LaunchShape> cand = candidates(kind, static_cast<int>(b));
    long long* dres = nullptr;
    if (cudaMalloc(&dres, 32) != cudaSuccess) return shapes_fail(SCAN_ENOMEM, "cudaMalloc(result) failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);

    Entry saved;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        saved = g_table[kind][b];
    }
    auto install = [&](const gb::LaunchShape* s) {
        std::lock_guard<std::mutex> lock(g_mu);
        Entry& e = g_table[kind][b];
        if (s) {
            e.tuned = true;
            e.shape = *s;
        } else {
            e = Entry{};
        }
    };
    scan_status status = SCAN_OK;
    // mean time of `k` back-to-back scans with shape s (nullptr: the rule)
    auto time_shape = [&](const gb::LaunchShape* s, uint32_t k, float* us) -> scan_status {
        install(s);
        bool empty = false;
        scan_status r = gb_enqueue_scan(col, pred, strategy, st, dres, &empty);  // warm-up
        if (r != SCAN_OK) return r;
        if (empty) return shapes_fail(SCAN_EINVAL, "the predicate selects nothing: tune with a non-empty range");
        cudaEventRecord(e0, st);
        for (uint32_t i = 0; i < k && r == SCAN_OK; ++i) r = gb_enqueue_scan(col, pred, strategy, st, dres, &empty);
        cudaEventRecord(e1, st);
        if (r != SCAN_OK) return r;
        if (cudaEventSynchronize(e1) != cudaSuccess) return shapes_fail(SCAN_ECUDA, "a tuning launch failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *us = ms * 1000.f / static_cast<float>(k);
        return SCAN_OK;
    };

    std::vector<float> t(cand.size(), 0.f);
    for (size_t i = 0; i < cand.size() && status == SCAN_OK; ++i) status = time_shape(&cand[i], reps, &t[i]);
    float def_us = 0.f, best_us = 0.f;
    size_t best = 0;
    if (status == SCAN_OK) {
        // re-time the three fastest and the rule, interleaved, with more repetitions
        std::vector<size_t> order(cand.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return t[x] < t[y]; });
        order.resize(std::min<size_t>(order.size(), 3));
        std::vector<float> acc(order.size(), 0.f);
        float acc_def = 0.f;
        for (int round = 0; round < 3 && status == SCAN_OK; ++round) {
            float us = 0.f;
            status = time_shape(nullptr, 2 * reps, &us);
            acc_def += us;
            for (size_t j = 0; j < order.size() && status == SCAN_OK; ++j) {
                status = time_shape(&cand[order[j]], 2 * reps, &us);
                acc[j] += us;
            }
        }
        if (status == SCAN_OK) {
            def_us = acc_def / 3.f;
            size_t bj = 0;
            for (size_t j = 1; j < acc.size(); ++j)
                if (acc[j] < acc[bj]) bj = j;
            best = order[bj];
            best_us = acc[bj] / 3.f;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dres);
    if (status != SCAN_OK) {
        std::lock_guard<std::mutex> lock(g_mu);
        g_table[kind][b] = saved;
        return status;
    }
    {
        std::lock_guard<std::mutex> lock(g_mu);
        Entry& e = g_table[kind][b];
        const bool win = best_us < def_us;
        e.tuned = win;
        e.shape = win ? cand[best] : default_shape(kind, static_cast<int>(b));
        e.best_us = win ? best_us : def_us;
        e.default_us = def_us;
        out->best = to_abi(e.shape);
    }
    out->rule = to_abi(default_shape(kind, static_cast<int>(b)));
    out->best_us = best_us < def_us ? best_us : def_us;
    out->rule_us = def_us;
    out->candidates = static_cast<uint32_t>(cand.size());
    return SCAN_OK;
}

scan_status scan_autotune_save(const char* path)
{
    gb_set_last_error("");
    if (!path) return shapes_fail(SCAN_EINVAL, "path is NULL");
    std::string text = std::string(kMagic) + " " + std::to_string(kVersion) + "\n";
    text += "device " + device_identity() + "\n";
    text += "# kind b warps stages tile_blocks vote_rows vec_lanes tuned_us rule_us\n";
    {
        std::lock_guard<std::mutex> lock(g_mu);
        for (int k = 0; k < kKinds; ++k)
            for (int b = 1; b <= 32; ++b) {
                const Entry& e = g_table[k][b];
                if (!e.tuned) continue;
                char line[160];
                std::snprintf(line, sizeof line, "%s %d %d %d %d %d %d %.3f %.3f\n", kKindName[k], b, e.shape.warps,
                              e.shape.stages, e.shape.tile_blocks, e.shape.vote_rows, e.shape.vec_lanes, e.best_us,
                              e.default_us);
                text += line;
            }
    }
    FILE* f = std::fopen(path, "w");
    if (!f) return shapes_fail(SCAN_EINVAL, std::string("cannot write ") + path + ": " + std::strerror(errno));
    const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
    if (std::fclose(f) != 0 || !ok) return shapes_fail(SCAN_EINVAL, std::string("cannot write ") + path);
    return SCAN_OK;
}

scan_status scan_autotune_load(const char* path)
{
    gb_set_last_error("");
    if (!path) return shapes_fail(SCAN_EINVAL, "path is NULL");
    FILE* f = std::fopen(path, "r");
    if (!f) return shapes_fail(SCAN_EINVAL, std::string("cannot read ") + path + ": " + std::strerror(errno));
    std::vector<std::string> lines;
    char buf[512];
    while (std::fgets(buf, sizeof buf, f)) {
        std::string s = buf;
        if (!s.empty() && s.back() != '\n' && !std::feof(f)) {
            std::fclose(f);
            return shapes_fail(SCAN_EINVAL, "line too long in the shape cache");
        }
        while (!s.empty() && (s.back() == '\n' || s.back() == '\r')) s.pop_back();
        lines.push_back(s);
    }
    std::fclose(f);
    auto bad = [&](size_t i, const std::string& why) {
        return shapes_fail(SCAN_EINVAL, "shape cache line " + std::to_string(i + 1) + ": " + why);
    };
    char magic[32];
    int version = 0;
    if (lines.empty() || std::sscanf(lines[0].c_str(), "%31s %d", magic, &version) != 2 ||
        std::strcmp(magic, kMagic) != 0)
        return bad(0, "not a gbscan shape cache");
    if (version != kVersion)
        return bad(0, "version " + std::to_string(version) + " (this library reads " + std::to_string(kVersion) + ")");
    if (lines.size() < 2 || lines[1].rfind("device ", 0) != 0) return bad(1, "missing the device line");
    const std::string want = device_identity();
    if (lines[1].substr(7) != want)
        return bad(1, "tuned on '" + lines[1].substr(7) + "', this device is '" + want + "'");
    Entry fresh[kKinds][33];
    for (size_t i = 2; i < lines.size(); ++i) {
        const std::string& s = lines[i];
        if (s.empty() || s[0] == '#') continue;
        char kname[32];
        int b, w, st, tb, v, vl, used = 0;
        float tu, ru;
        if (std::sscanf(s.c_str(), "%31s %d %d %d %d %d %d %f %f%n", kname, &b, &w, &st, &tb, &v, &vl, &tu, &ru,
                        &used) != 9 ||
            s.find_first_not_of(" \t", static_cast<size_t>(used)) != std::string::npos)
            return bad(i, "expected: kind b warps stages tile_blocks vote_rows vec_lanes tuned_us rule_us");
        int kind = -1;
        for (int k = 0; k < kKinds; ++k)
            if (std::strcmp(kname, kKindName[k]) == 0) kind = k;
        if (kind < 0) return bad(i, std::string("unknown kernel kind '") + kname + "'");
        const gb::LaunchShape shape{w, st, tb, v, vl};
        const char* why = nullptr;
        if (!shape_ok(kind, b, shape, &why)) return bad(i, why);
        if (fresh[kind][b].tuned) return bad(i, "duplicate entry");
        fresh[kind][b].tuned = true;
        fresh[kind][b].shape = shape;
        fresh[kind][b].best_us = tu;
        fresh[kind][b].default_us = ru;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    for (int k = 0; k < kKinds; ++k)
        for (int b = 0; b <= 32; ++b) g_table[k][b] = fresh[k][b];
    return SCAN_OK;
}

}  // extern "C"
