// Checked builds (the library compiled with -DFDAS_CHECK_BOUNDS, built as
// libfdas_checked.so): device-side bounds checks written as error records.
//
// FDAS_IN_BOUNDS(begin, count, limit, site) is true when the elements
// [begin, begin + count) lie inside [0, limit).  In a checked build a check
// that fails records itself in its translation unit's log (the number of
// failed checks; site, range and limit of the first) and evaluates to false,
// and the code skips the access it guards: a bad index neither faults the GPU
// nor traps, and the kernel runs to its end (every barrier still gets its
// arrivals).  The host reads and clears the logs after each launch group
// (plan.cu) and turns a failure into FDAS_ERR_BOUNDS.  In ordinary builds the
// macro is the constant true, its arguments are not compiled, and the kernels
// are exactly the unchecked ones.
//
// Kernels whose limits are not among their arguments take one more argument
// in checked builds only: FDAS_BC_PARAM in the parameter list, FDAS_BC_ARG(...)
// at the launch (up to four int64 limits, read as bc.lim[i]).
//
// Fault injection for tests: FDAS_FAULT=bounds (checked builds) lowers every
// limit by g_bounds_shrink elements for one search, so that checks fail at
// real sites while the accesses they skip were in fact in bounds.
#pragma once

#include <stdint.h>

namespace fdas {

enum BoundsSite : int32_t {
    kSiteNone = 0,
    kSiteHsSpanRow,        // harmonic sum: source row of a span copy
    kSiteHsSpanRange,      // harmonic sum: span copy inside its row
    kSiteHsTopLoad,        // harmonic sum: the thread's top-row cells
    kSiteHsSumsStore,      // harmonic sums output
    kSiteFundRow,          // fundamental-indexed sum: row of harmonic k
    kSiteFundRun,          // fundamental-indexed sum: run of harmonic k in its row
    kSiteSortRecord,       // candidate ordering: record index
    kSiteTcImageCopy,      // tensor-core correlation: template image copy (global)
    kSiteTcImageSmem,      // tensor-core correlation: template image size (shared)
    kSiteTcWindowCopy,     // tensor-core correlation: spectrum window copy
    kSiteTcWindowRead,     // tensor-core correlation: MMA rows inside the window
    kSiteTcEnergy,         // tensor-core correlation: template energy index
    kSiteTcPlaneStore,     // tensor-core correlation: plane / F store
    kSiteTcEdgeStore,      // tensor-core correlation: interbinning edge table
    kSiteCount
};

__host__ __device__ inline const char *bounds_site_name(int32_t s) {
    switch (s) {
        case kSiteHsSpanRow: return "harmonic sum: source row of a span copy";
        case kSiteHsSpanRange: return "harmonic sum: span copy inside its row";
        case kSiteHsTopLoad: return "harmonic sum: top-row cells of a thread";
        case kSiteHsSumsStore: return "harmonic sums: output store";
        case kSiteFundRow: return "fundamental-indexed sum: row of a harmonic";
        case kSiteFundRun: return "fundamental-indexed sum: run inside its row";
        case kSiteSortRecord: return "candidate ordering: record index";
        case kSiteTcImageCopy: return "tensor-core correlation: template image copy";
        case kSiteTcImageSmem: return "tensor-core correlation: template image in shared memory";
        case kSiteTcWindowCopy: return "tensor-core correlation: spectrum window copy";
        case kSiteTcWindowRead: return "tensor-core correlation: MMA rows inside the window";
        case kSiteTcEnergy: return "tensor-core correlation: template energy";
        case kSiteTcPlaneStore: return "tensor-core correlation: plane store";
        case kSiteTcEdgeStore: return "tensor-core correlation: interbinning edge store";
        default: return "unknown site";
    }
}

// the first failed check of a translation unit, and how many failed
struct BoundsLog {
    unsigned long long failures;
    int32_t site;
    int32_t pad;
    int64_t begin, count, limit;
};

struct BoundsCtx {
    int64_t lim[4];
};

#ifdef FDAS_CHECK_BOUNDS

static __device__ BoundsLog g_bounds_log;
static __device__ int64_t g_bounds_shrink;

__device__ __forceinline__ bool bounds_ok(int64_t begin, int64_t count, int64_t limit,
                                          int32_t site) {
    const int64_t lim = limit - g_bounds_shrink;
    if (begin >= 0 && count >= 0 && begin <= lim - count) return true;
    if (atomicAdd(&g_bounds_log.failures, 1ull) == 0ull) {
        g_bounds_log.site = site;
        g_bounds_log.begin = begin;
        g_bounds_log.count = count;
        g_bounds_log.limit = limit;
    }
    return false;
}

#define FDAS_IN_BOUNDS(begin, count, limit, site)                                     \
    ::fdas::bounds_ok((int64_t)(begin), (int64_t)(count), (int64_t)(limit), (site))
#define FDAS_BC_PARAM , ::fdas::BoundsCtx bc
#define FDAS_BC_ARG(...) , ::fdas::BoundsCtx{{__VA_ARGS__}}

// host side of a translation unit's log: bounds_take_<tu> copies the log out
// (after the device is idle) and clears it; bounds_arm_<tu> sets the shrink
#define FDAS_BOUNDS_LOG_TU(tu)                                                          \
    cudaError_t bounds_take_##tu(BoundsLog *out) {                                      \
        cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_log, sizeof(BoundsLog));     \
        if (e != cudaSuccess) return e;                                                 \
        const BoundsLog zero{};                                                         \
        return cudaMemcpyToSymbol(g_bounds_log, &zero, sizeof(BoundsLog));              \
    }                                                                                   \
    cudaError_t bounds_arm_##tu(int64_t shrink) {                                       \
        return cudaMemcpyToSymbol(g_bounds_shrink, &shrink, sizeof(int64_t));           \
    }

#else

#define FDAS_IN_BOUNDS(begin, count, limit, site) true
#define FDAS_BC_PARAM
#define FDAS_BC_ARG(...)
#define FDAS_BOUNDS_LOG_TU(tu)

#endif

}  // namespace fdas
