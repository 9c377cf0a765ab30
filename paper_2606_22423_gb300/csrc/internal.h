// Host-side declarations shared between the library's translation units
// (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/gbscan.h"

// Sets the message scan_last_error() returns on this thread.
void gb_set_last_error(const char* msg);

// SM count and cooperative-launch support of the current device (cached per device).
int gb_device_sms();
bool gb_device_coop();

// Read-only view of a column.
bool gb_column_view(const scan_column* c, const uint32_t** packed, uint64_t* n, uint32_t* b,
                    uint32_t* base, const uint2** zonemap);

// Workspace of the materializing select on one column.
struct GbSelectWs {
    unsigned long long* agg;   // tagged per-iteration CTA totals
    uint32_t epoch;            // this launch's tag
    unsigned int* status;      // the column's device status word
    long long* result;         // the column's device result slot (4 words, status follows)
    scan_result* host_result;  // pinned staging for result + status (36 bytes)
};

// The column's selection-vector buffer for conjunctive scans, grown to at
// least `words` 32-bit words (kept for later calls; freed with the column).
cudaError_t gb_column_conj_mask(scan_column* c, uint64_t words, uint32_t** out);

// Grows the column's select workspace to at least `words` tagged words and
// hands out a fresh tag (clearing the words when the tag wraps).
cudaError_t gb_column_select_ws(scan_column* c, uint64_t words, cudaStream_t st, GbSelectWs* out);

namespace gb {
struct ScanParams;
struct LaunchShape;
}
// Launch shape of kernel `op` (gb::OpKind) at width b: the installed tuned
// shape for the four tunable scan kernels, else the built-in rule.
gb::LaunchShape gb_shape_for(int b, int op);

// The tuner's candidate shapes for (op, b), and installing one (nullptr: the
// rule again); false for an illegal shape.
std::vector<gb::LaunchShape> gb_shape_candidates(int b, int op);
bool gb_shape_install(int b, int op, const gb::LaunchShape* shape, float tuned_us, float rule_us);

// Enqueues one scan of `c` (what scan_run_async does, with the result written
// to dev_result); *empty is set when the predicate selects nothing and no
// kernel was launched.
scan_status gb_enqueue_scan(scan_column* c, scan_pred pred, scan_strategy strategy, cudaStream_t st,
                            long long* dev_result, bool* empty);
// Scan parameters of a column: its packed data, n, base, zone map and device
// workspace (result, status, grid-finish ticket, queue counters, partials).
gb::ScanParams gb_column_params(const scan_column* c);
