// semr_reduce_async_noalloc: the reduction for callers that cannot allocate
// device memory.  The fused kernel needs scratch (the look-back tile states
// and the per-tile norm partials); here it comes from one file-scope device
// array instead of a caller buffer or an allocation.  The paper has no
// counterpart to this entry point.
#include <cuda_runtime.h>

#include <mutex>

#include "semr_internal.h"

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) uint8_t g_semr_noalloc_scratch[SEMR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SEMR_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_semr_noalloc_scratch) != cudaSuccess || !p) return SEMR_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SEMR_OK;
}

}  // namespace

extern "C" int semr_reduce_async_noalloc(const semr_fieldset* fs, const semr_mesh* mesh, uint8_t* payload,
                                         uint64_t payload_cap, double* elem_report, semr_summary* summary,
                                         void* cuda_stream) {
    if (!fs || !mesh) return SEMR_EINVAL;
    semr_sizes sz;
    int rc = semr_sizes_for(mesh->lx, mesh->n_elem, fs->n_fields, fs->tau, &sz);
    if (rc) return rc;
    // beyond the fixed scratch (it may hold less than the recommended size: the lx = 8 kernel
    // then runs on as many CTAs as the array can stage codes for)
    if (semr::scratch_min(mesh->lx, mesh->n_elem, fs->n_fields) > SEMR_NOALLOC_SCRATCH_BYTES) return SEMR_EBUDGET;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc) return rc;
    semr_outputs o;
    o.payload = payload;
    o.payload_cap = payload_cap;
    o.elem_report = elem_report;
    o.summary = summary;
    o.scratch = scratch;
    o.scratch_bytes = SEMR_NOALLOC_SCRATCH_BYTES;
    return semr_reduce_async(fs, mesh, &o, cuda_stream);
}
