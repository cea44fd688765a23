// Bounds-checking build (-DHELM_CHECK_BOUNDS): the global-memory accesses of the
// kernels that go through HELM_CHK (every bulk copy, and the computed loads and stores
// of the stage, interface, Krylov and HABC kernels) first check that the bytes they
// touch lie inside one live device range: an allocation of the library or a buffer
// of the current call.  A failed check counts the violation, records the first one
// (address, size, source line) and skips the access, so a bad index shows up as a
// report (helm_check_bounds_report) instead of a fault.
//
// Each translation unit keeps its own copy of the range table in device memory (the
// library is built without relocatable device code); the host uploads the same table
// to every unit whenever it changes.  In the normal build HELM_CHK(p, bytes) is the
// constant true and none of this is compiled.
#pragma once

#include <cuda_runtime.h>

constexpr int HC_MAX_RANGES = 384;

struct HcRange {
    unsigned long long lo, hi;       // [lo, hi)
};
struct HcTable {
    int n;
    HcRange r[HC_MAX_RANGES];
};
struct HcBad {
    unsigned long long count;        // failed checks
    unsigned long long addr, bytes;  // the first one
    int line;
    int unit;                        // index of the translation unit (set by the host)
};

// per-unit uploader of the range table, reader and reset of the violation record
// (registered at library load)
using HcUpload = cudaError_t (*)(const HcTable&);
using HcRead = cudaError_t (*)(HcBad&);
using HcReset = cudaError_t (*)();
void hc_register_unit(HcUpload up, HcRead rd, HcReset rs, const char* file);

#ifdef HELM_CHECK_BOUNDS
namespace {
__device__ HcTable hc_table;
__device__ HcBad hc_bad;

__device__ __noinline__ bool hc_ok(const void* p, unsigned long long bytes, int line) {
    const unsigned long long a = reinterpret_cast<unsigned long long>(p), b = a + bytes;
    const int n = hc_table.n;
    for (int i = 0; i < n; ++i)
        if (a >= hc_table.r[i].lo && b <= hc_table.r[i].hi) return true;
    if (atomicAdd(&hc_bad.count, 1ull) == 0ull) {
        hc_bad.addr = a;
        hc_bad.bytes = bytes;
        hc_bad.line = line;
    }
    return false;
}

cudaError_t hc_upload_unit(const HcTable& t) { return cudaMemcpyToSymbol(hc_table, &t, sizeof(HcTable)); }
cudaError_t hc_read_unit(HcBad& b) { return cudaMemcpyFromSymbol(&b, hc_bad, sizeof(HcBad)); }
cudaError_t hc_reset_unit() {
    const HcBad z{};
    return cudaMemcpyToSymbol(hc_bad, &z, sizeof(HcBad));
}

struct HcUnitRegistration {
    HcUnitRegistration() { hc_register_unit(&hc_upload_unit, &hc_read_unit, &hc_reset_unit, __BASE_FILE__); }
} hc_unit_registration;
}  // namespace

#define HELM_CHK(p, bytes) hc_ok((p), (unsigned long long)(bytes), __LINE__)
#else
#define HELM_CHK(p, bytes) true
#endif

// checked element access: a failed check reads zero and drops the store
template <typename T> __device__ __forceinline__ T hc_load(const T* p, bool ok) { return ok ? *p : T{}; }
template <typename T> __device__ __forceinline__ T hc_loadcg(const T* p, bool ok) { return ok ? __ldcg(p) : T{}; }
#define HLD(p) hc_load((p), HELM_CHK((p), sizeof(*(p))))
#define HLDCG(p) hc_loadcg((p), HELM_CHK((p), sizeof(*(p))))
#define HST(p, v)                                   \
    do {                                            \
        if (HELM_CHK((p), sizeof(*(p)))) *(p) = (v); \
    } while (0)
