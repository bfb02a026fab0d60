// Bounds checks of the checked build.  Compiled with -DHC_CHECK (the library
// libhc_check.so), every checked device access first tests its index against
// its bound; an index out of range is counted, the first one is recorded
// (site, index, bound) and the access is skipped, so a faulty index shows up
// in hc_check_status instead of touching memory it does not own.  In the
// normal build HC_IN_BOUNDS is the constant true and its arguments are not
// evaluated.
//
// Each translation unit keeps its own record (a static __device__ variable)
// and registers a host reader for it at load time; hc_check_status (api.cu)
// folds them together.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hc {

// Check sites (hc_check_report.site, documented in include/hc.h).
enum CheckSite : uint32_t {
    kSiteNone = 0,
    kSiteKeySlot = 1,       // key pass: the row's slot in its list
    kSiteScatter = 2,       // radix scatter: a record's destination in its segment
    kSiteRunList = 3,       // run fix-up: the list of run starts
    kSiteRunWrite = 4,      // run fix-up: a record's place in its run
    kSiteLongRun = 5,       // long-run pass: a record's place in the pass output
    kSiteSearch = 6,        // lower_bound: a probed entry of the list
    kSiteWindow = 7,        // window end against the list length
    kSiteEntry = 8,         // a window entry against the index's entries
    kSiteRow = 9,           // a row id against the database rows
    kSiteQuery = 10,        // a query number against the batch
    kSiteMultiQuery = 11,   // persistent launch: a query of a job
    kSiteMultiLists = 12,   // persistent launch: lists of a job's index
    kSitePad = 13,          // a guard pad behind a library buffer was overwritten
};

struct CheckRecord {
    unsigned long long count;   // accesses refused
    uint32_t site;              // first refused access
    uint32_t pad;
    unsigned long long index, bound;
};

// Host reader of one translation unit's record (reset: clear it after reading).
using CheckReader = int (*)(CheckRecord* out, bool reset);
// Adds a reader (api.cu); called while the library loads.
void register_check_reader(CheckReader r);

#ifdef HC_CHECK

static __device__ CheckRecord g_check_record;

__device__ __forceinline__ bool check_index(uint32_t site, uint64_t i, uint64_t n) {
    if (i < n) return true;
    if (atomicAdd(&g_check_record.count, 1ull) == 0ull) {
        g_check_record.site = site;
        g_check_record.index = i;
        g_check_record.bound = n;
    }
    return false;
}

#define HC_IN_BOUNDS(site, i, n) (::hc::check_index((site), (uint64_t)(i), (uint64_t)(n)))

static int read_check_record(CheckRecord* out, bool reset) {
    if (cudaMemcpyFromSymbol(out, g_check_record, sizeof(CheckRecord)) != cudaSuccess) return -3;
    if (reset) {
        const CheckRecord z{};
        if (cudaMemcpyToSymbol(g_check_record, &z, sizeof(CheckRecord)) != cudaSuccess) return -3;
    }
    return 0;
}
static const int g_check_registered = (register_check_reader(&read_check_record), 0);

#else

#define HC_IN_BOUNDS(site, i, n) true

#endif

}  // namespace hc
