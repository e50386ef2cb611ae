// Trap-free index checks of the debug build (compiled with -DGDG_CHECKS=1,
// built as libgdg_checks.so by build.build(checks=True)).
//
// Every place where a kernel derives an element index from another one (the
// face neighbours of the stage kernels, the neighbour blocks of the
// persistent step, the work items of the batched launch) checks it against
// the range of elements the buffers hold.  A failed check never traps: it
// counts the failure, records the first one (site, index, bound) in a
// device-side slot and replaces the index by a valid one, so the kernel
// finishes and the host reads the record (gdg_check_status).  The ordinary
// build compiles the checks to nothing.
//
// Without relocatable device code every translation unit has its own slot;
// each one that includes this header defines its reader with
// GDG_CHECKS_READER(name), and gdg_check_status sums them.
#pragma once

#include <cuda_runtime.h>

#ifndef GDG_CHECKS
#define GDG_CHECKS 0
#endif

// check sites (the record names the first failing one)
enum GdgCheckSite {
    GDG_SITE_STAGE2P_NB = 1,      // + 0..3: x-, x+, y-, y+ neighbour of the one-line modal body
    GDG_SITE_STAGE2H_NB = 5,      // + 0..3: the half-line body
    GDG_SITE_STAGE2_NB = 9,       // + 0..3: the generic 2-D stage
    GDG_SITE_STAGE2F_NB = 13,     // + 0..3: the field-split stage
    GDG_SITE_STAGE2R_NB = 17,     // + 0..3: the persistent step
    GDG_SITE_STEP2R_BLOCK = 21,   // a neighbour block of the persistent step
    GDG_SITE_STAGE1_NB = 22,      // + 0..1: the 1-D stage
    GDG_SITE_STAGE3_NB = 30,      // + 0..5: the 3-D stages (x-, x+, y-, y+, z-, z+)
    GDG_SITE_VAR_NB = 40,         // the face neighbour of a variable-coefficient element
    GDG_SITE_BATCH_PROBLEM = 50,  // the problem of a batched work item
    GDG_SITE_BATCH_ELEMENT = 51,  // the element (or modal tile) of a batched work item
    GDG_SITE_SELFTEST = 99,       // gdg_check_selftest
};

struct GdgCheckSlot {
    unsigned long long count;
    long long site, index, bound;
};

#if defined(__CUDACC__)   // device side and readers: CUDA translation units only
#if GDG_CHECKS
namespace {
__device__ GdgCheckSlot g_gdg_check_slot;
}

// true when lo <= i < hi; otherwise counts and (first failure) records
__device__ __forceinline__ bool gdg_in_range(long long i, long long lo, long long hi, int site) {
    if (i >= lo && i < hi) return true;
    if (atomicAdd(&g_gdg_check_slot.count, 1ull) == 0ull) {
        g_gdg_check_slot.site = site;
        g_gdg_check_slot.index = i;
        g_gdg_check_slot.bound = i < lo ? lo : hi;
    }
    return false;
}
#define GDG_CHECK_INDEX(i, lo, hi, site, fallback)                                 \
    do {                                                                           \
        if (!gdg_in_range((long long)(i), (long long)(lo), (long long)(hi), (site))) \
            (i) = (fallback);                                                      \
    } while (0)

// host reader of this translation unit's slot (reset: zero it after reading)
#define GDG_CHECKS_READER(name)                                                                \
    int name(GdgCheckSlot *out, int reset) {                                                   \
        GdgCheckSlot s{};                                                                      \
        if (cudaMemcpyFromSymbol(&s, g_gdg_check_slot, sizeof(s)) != cudaSuccess) return -1;   \
        if (reset) {                                                                           \
            const GdgCheckSlot z{};                                                            \
            if (cudaMemcpyToSymbol(g_gdg_check_slot, &z, sizeof(z)) != cudaSuccess) return -1; \
        }                                                                                      \
        *out = s;                                                                              \
        return 0;                                                                              \
    }
#else
#define GDG_CHECK_INDEX(i, lo, hi, site, fallback) \
    do {                                           \
    } while (0)
#define GDG_CHECKS_READER(name)                    \
    int name(GdgCheckSlot *out, int) {             \
        *out = GdgCheckSlot{};                     \
        return 0;                                  \
    }
#endif
#endif   // __CUDACC__

// the element range of a 2-D modal problem's trace buffer (ghost rows of a
// band of a partitioned mesh included)
#define GDG_CHECK_ELEM2(f, mp, site)                                                                      \
    GDG_CHECK_INDEX(f, (mp).halo_lo ? -(long long)(mp).nx : 0LL,                                          \
                    (long long)(mp).ne + ((mp).halo_hi ? (long long)(mp).nx : 0LL), site, 0)

// readers of the translation units (gdg_check_status sums them; the batch
// reader sums its three budgets' translation units)
int gdg_checks_read_const(GdgCheckSlot *out, int reset);
int gdg_checks_read_const3(GdgCheckSlot *out, int reset);
int gdg_checks_read_var(GdgCheckSlot *out, int reset);
int gdg_checks_read_batch(GdgCheckSlot *out, int reset);
