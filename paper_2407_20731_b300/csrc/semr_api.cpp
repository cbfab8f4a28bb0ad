// C-ABI runtime of libsemr: argument validation, buffer sizing, launches of
// the fused reduce kernel, the ticketed stream API with a device-memory
// budget, and the host-side payload decoder.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "semr_internal.h"

using namespace semr;

namespace {

bool lx_supported(int lx) { return lx >= SEMR_LX_MIN && lx <= SEMR_LX_MAX; }

int check_common(int32_t lx, int64_t n_elem, int32_t n_fields, double tau) {
    if (!lx_supported(lx)) return SEMR_EINVAL;
    if (n_elem < 1 || n_fields < 1 || n_fields > SEMR_MAX_FIELDS) return SEMR_EINVAL;
    const uint64_t n3 = uint64_t(lx) * lx * lx;
    if (uint64_t(n_elem) * n3 >= (1ull << 40)) return SEMR_EINVAL;
    if (!(tau >= 0.0) || std::isinf(tau)) return SEMR_EINVAL;
    // a kept code is at most 2/sqrt(tau) in magnitude: below 2^-60 it would not fit int32;
    // above 2^64 nothing can be kept (a_m^2 <= S_e) and t = tau S_e may leave the range
    if (tau != 0.0 && (tau <= 0x1p-60 || tau > 0x1p64)) return SEMR_EINVAL;
    return SEMR_OK;
}

uint64_t tiles_per_field(int lx, int64_t n_elem) {
    const int t = tile_elems(lx);
    return (uint64_t(n_elem) + t - 1) / t;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Scratch of one reduction: the CTA kernels' layout, and at lx = 8 also the
// warp kernel's (whichever of the two runs, the buffer holds it).
uint64_t semr::scratch_need(int lx, int64_t n_elem, int32_t n_fields) {
    const uint64_t cta = scratch_bytes(uint64_t(n_fields) * tiles_per_field(lx, n_elem));
    if (lx == 8) return std::max(cta, warp_scratch_bytes(n_elem, n_fields));
    if (group_tile(lx)) return std::max(cta, warp_scratch_bytes(n_elem, n_fields, group_tile(lx)));
    return cta;
}
uint64_t semr::scratch_min(int lx, int64_t n_elem, int32_t n_fields) {
    const uint64_t cta = scratch_bytes(uint64_t(n_fields) * tiles_per_field(lx, n_elem));
    if (lx == 8) return std::max(cta, warp_scratch_min(n_elem, n_fields));
    if (group_tile(lx)) return std::max(cta, warp_scratch_min(n_elem, n_fields, group_tile(lx)));
    return cta;
}

extern "C" int semr_sizes_for(int32_t lx, int64_t n_elem, int32_t n_fields, double tau, semr_sizes* out) {
    if (!out) return SEMR_EINVAL;
    int rc = check_common(lx, n_elem, n_fields, tau);
    if (rc) return rc;
    const uint64_t n3 = uint64_t(lx) * lx * lx;
    const int width = code_width(tau);
    const uint64_t tiles = uint64_t(n_fields) * tiles_per_field(lx, n_elem);
    out->header_bytes = header_bytes(n_fields);
    out->code_base = out->header_bytes + uint64_t(n_fields) * field_fixed_bytes(lx, n_elem);
    out->payload_worst = out->code_base + uint64_t(width) * n3 * uint64_t(n_elem) * n_fields;
    out->scratch_bytes = scratch_need(lx, n_elem, n_fields);
    out->elem_report_bytes = 24ull * uint64_t(n_elem) * n_fields;
    out->code_width = (uint32_t)width;
    out->tiles = (uint32_t)std::min<uint64_t>(tiles, 0xffffffffull);
    out->scratch_min_bytes = scratch_min(lx, n_elem, n_fields);
    return SEMR_OK;
}

#ifdef SEMR_BOUNDS
// semr_selftest_bounds only: launch with a payload capacity this many bytes short of the fixed
// sections (inside a buffer that holds them all), so the kernels' range tests must fail
static uint64_t g_bounds_cap_short = 0;
#endif

extern "C" int semr_reduce_async(const semr_fieldset* fs, const semr_mesh* mesh, const semr_outputs* out,
                                 void* cuda_stream) {
    return semr_reduce_async_timed(fs, mesh, out, cuda_stream, nullptr, nullptr);
}

extern "C" int semr_reduce_async_timed(const semr_fieldset* fs, const semr_mesh* mesh, const semr_outputs* out,
                                       void* cuda_stream, void* ev_begin, void* ev_end) {
    if (!fs || !mesh || !out) return SEMR_EINVAL;
    if (mesh->lx >= 2 && !lx_supported(mesh->lx)) return SEMR_EUNSUPPORTED;
    int rc = check_common(mesh->lx, mesh->n_elem, fs->n_fields, fs->tau);
    if (rc) return rc;
    if (fs->precision != SEMR_FP64 && fs->precision != SEMR_FP32 && fs->precision != SEMR_FP64_NATIVE)
        return SEMR_EUNSUPPORTED;
    if (fs->flags & ~(SEMR_WRITE_RECON | SEMR_CUMULATIVE)) return SEMR_EINVAL;
    const bool cumulative = (fs->flags & SEMR_CUMULATIVE) && fs->tau != 0.0;
    if (cumulative && fs->precision == SEMR_FP64_NATIVE) return SEMR_EUNSUPPORTED;
    if (!mesh->jac || !out->payload || !out->summary || !out->scratch) return SEMR_EINVAL;
    if ((reinterpret_cast<uintptr_t>(out->scratch) & 255u) != 0 || !aligned16(out->payload)) return SEMR_EINVAL;
    // even lx: element blocks are loaded as 16-byte vectors; odd lx: 8-byte scalars
    const uintptr_t amask = (mesh->lx % 2 == 0) ? 15u : 7u;
    for (int f = 0; f < fs->n_fields; ++f) {
        if (!fs->fields[f] || (reinterpret_cast<uintptr_t>(fs->fields[f]) & amask)) return SEMR_EINVAL;
        if ((fs->flags & SEMR_WRITE_RECON) && fs->recon[f] && (reinterpret_cast<uintptr_t>(fs->recon[f]) & 7u))
            return SEMR_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(mesh->jac) & 7u) return SEMR_EINVAL;
    semr_sizes sz;
    semr_sizes_for(mesh->lx, mesh->n_elem, fs->n_fields, fs->tau, &sz);
    if (out->scratch_bytes < scratch_min(mesh->lx, mesh->n_elem, fs->n_fields) || out->payload_cap < sz.code_base)
        return SEMR_EINVAL;

    LaunchParams p;
    std::memset(&p, 0, sizeof(p));
    for (int f = 0; f < fs->n_fields; ++f) {
        p.fields[f] = fs->fields[f];
        p.recon[f] = (fs->flags & SEMR_WRITE_RECON) ? fs->recon[f] : nullptr;
    }
    p.jac = mesh->jac;
    p.payload = out->payload;
    p.payload_cap = out->payload_cap;
    p.elem_report = out->elem_report;
    p.summary = out->summary;
    const uint64_t tiles = uint64_t(fs->n_fields) * tiles_per_field(mesh->lx, mesh->n_elem);
    split_scratch(p, static_cast<uint8_t*>(out->scratch), tiles);
    p.lx = mesh->lx;
    p.tile = tile_elems(mesh->lx);
    p.n_elem = mesh->n_elem;
    p.n_fields = fs->n_fields;
    p.tiles_per_field = (int32_t)tiles_per_field(mesh->lx, mesh->n_elem);
    p.tau = fs->tau;
    p.lossless = fs->tau == 0.0;
    p.width = (int32_t)sz.code_width;
    p.write_recon = (fs->flags & SEMR_WRITE_RECON) ? 1 : 0;
    p.precision = fs->precision;
    p.cumulative = cumulative ? 1 : 0;
    p.header_bytes = sz.header_bytes;
    p.fixed_bytes = field_fixed_bytes(mesh->lx, mesh->n_elem);
    p.code_base = sz.code_base;
#ifdef SEMR_BOUNDS
    if (g_bounds_cap_short) p.payload_cap = p.code_base - g_bounds_cap_short;
#endif
    // threshold truncation with int16 codes runs on the warp-level kernels: lx = 8 on the
    // warp-per-element kernel, lx = 6 and 10 on the warp-group kernel
    const bool warp = warp_applicable(p);
    const bool group = !warp && group_applicable(p);
    uint64_t zero = scratch_zero_bytes(tiles);
    if (warp || group) {
        const int tile = warp ? kWarpTile : group_tile(mesh->lx);
        split_scratch_warp(p, static_cast<uint8_t*>(out->scratch), out->scratch_bytes, mesh->n_elem, fs->n_fields, tile);
        p.tile = tile;
        p.tiles_per_field = (int32_t)((uint64_t(mesh->n_elem) + tile - 1) / tile);
        zero = scratch_zero_bytes(warp_tiles(mesh->n_elem, fs->n_fields, tile));
    }

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMemsetAsync(out->scratch, 0, zero, st) != cudaSuccess) return SEMR_ECUDA;
    if (ev_begin && cudaEventRecord(static_cast<cudaEvent_t>(ev_begin), st) != cudaSuccess) return SEMR_ECUDA;
    const int lr = warp ? launch_reduce_warp(p, st) : group ? launch_reduce_group(p, st) : launch_reduce(p, mesh->lx, st);
    if (lr != cudaSuccess) return SEMR_ECUDA;
    if (ev_end && cudaEventRecord(static_cast<cudaEvent_t>(ev_end), st) != cudaSuccess) return SEMR_ECUDA;
    // the warp-level kernels finalize in their last CTA; the CTA kernels have a finalize kernel
    if (!warp && !group && launch_finalize(p, mesh->lx, st) != cudaSuccess) return SEMR_ECUDA;
    return SEMR_OK;
}

// ------------------------------------------------------------ stream API
//
// A ticket owns one stream-ordered device allocation (payload | scratch |
// summary | element report).  The payload is sized for an estimate of the
// snapshot's codes, not for every mode kept (which would be about 14 times
// the payload of a 64^3 x 4 snapshot at tau = 1e-3): the estimate is twice
// the largest share of modes kept by the stream's completed tickets (1/16 of
// all modes before the first one), plus 4096 codes.  A ticket whose codes
// do not fit is re-run once at its exact size, which the first run reports
// (its counts and steps are complete; only the codes were not written).
// Each ticket's summary is copied to pinned host memory behind the kernels,
// so completion and its status are known without a device round trip.  No
// call holds the stream's lock across a device wait or a copy.

namespace {

uint64_t align256(uint64_t b) { return (b + 255) & ~uint64_t(255); }

constexpr int kPinnedChunk = 64;  // pinned summaries allocated together

}  // namespace

struct Ticket {
    uint8_t* dev = nullptr;   // payload | scratch | summary | elem report
    uint64_t bytes = 0;       // of dev (what the budget counts)
    uint64_t payload_cap = 0;
    uint64_t off_scratch = 0, off_summary = 0, off_elem = 0, scratch_bytes = 0;
    cudaEvent_t done = nullptr;
    semr_summary* host_sum = nullptr;  // pinned, written by the stream before `done`
    semr_fieldset fs{};        // the request, kept for a re-run at the exact size
    semr_mesh mesh{};
    uint64_t modes = 0;        // n_fields * n_elem * lx^3
    bool rerun = false;        // already re-run once
    bool busy = false;         // a fetch is waiting for or copying this ticket
};

struct semr_stream {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;  // device-to-host copies of fetched results
    uint64_t budget = 0;
    uint64_t in_flight = 0;
    uint64_t next_ticket = 1;
    double fill = 1.0 / 32;  // largest share of modes kept so far (the estimate is twice it: 1/16 at first)
    bool fill_seen = false;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::vector<semr_summary*> pinned_free;
    std::vector<semr_summary*> pinned_chunks;
    std::mutex mu;
};

namespace {

semr_summary* pinned_get(semr_stream* s) {  // with s->mu held
    if (s->pinned_free.empty()) {
        semr_summary* c = nullptr;
        if (cudaMallocHost(reinterpret_cast<void**>(&c), sizeof(semr_summary) * kPinnedChunk) != cudaSuccess)
            return nullptr;
        s->pinned_chunks.push_back(c);
        for (int k = kPinnedChunk - 1; k >= 0; --k) s->pinned_free.push_back(c + k);
    }
    semr_summary* p = s->pinned_free.back();
    s->pinned_free.pop_back();
    return p;
}

// Allocate a ticket's device block for a payload of `payload_cap` bytes and
// launch its reduction, the summary copy and the completion event (s->mu held).
int ticket_launch(semr_stream* s, Ticket& t, const semr_sizes& sz, uint64_t payload_cap) {
    t.payload_cap = payload_cap;
    t.off_scratch = align256(payload_cap);
    t.off_summary = align256(t.off_scratch + sz.scratch_bytes);
    t.off_elem = align256(t.off_summary + sizeof(semr_summary));
    t.bytes = align256(t.off_elem + sz.elem_report_bytes);
    t.scratch_bytes = sz.scratch_bytes;
    if (cudaMallocAsync(reinterpret_cast<void**>(&t.dev), t.bytes, s->stream) != cudaSuccess) {
        t.dev = nullptr;
        return SEMR_ENOMEM;
    }
    semr_outputs o;
    o.payload = t.dev;
    o.payload_cap = t.payload_cap;
    o.elem_report = reinterpret_cast<double*>(t.dev + t.off_elem);
    o.summary = reinterpret_cast<semr_summary*>(t.dev + t.off_summary);
    o.scratch = t.dev + t.off_scratch;
    o.scratch_bytes = t.scratch_bytes;
    int rc = semr_reduce_async(&t.fs, &t.mesh, &o, s->stream);
    if (rc == SEMR_OK && cudaMemcpyAsync(t.host_sum, o.summary, sizeof(semr_summary), cudaMemcpyDeviceToHost,
                                         s->stream) != cudaSuccess)
        rc = SEMR_ECUDA;
    if (rc == SEMR_OK && cudaEventRecord(t.done, s->stream) != cudaSuccess) rc = SEMR_ECUDA;
    if (rc != SEMR_OK) {
        cudaFreeAsync(t.dev, s->stream);
        t.dev = nullptr;
    }
    return rc;
}

void release(semr_stream* s, Ticket& t) {  // s->mu held
    if (t.dev) cudaFreeAsync(t.dev, s->stream);
    if (t.done) cudaEventDestroy(t.done);
    if (t.host_sum) s->pinned_free.push_back(t.host_sum);
    s->in_flight -= t.bytes;
    t.dev = nullptr;
    t.done = nullptr;
    t.host_sum = nullptr;
}

// State of a ticket (s->mu held): SEMR_OK when its results are final,
// SEMR_EAGAIN while its work runs (a ticket whose codes overflowed its first
// payload is re-run here at the exact size), SEMR_EBUDGET when that re-run
// does not fit the budget next to the other tickets in flight (their memory
// is freed only when they are fetched), or an error.
int ticket_state(semr_stream* s, Ticket& t) {
    const cudaError_t e = cudaEventQuery(t.done);
    if (e == cudaErrorNotReady) return SEMR_EAGAIN;
    if (e != cudaSuccess) return SEMR_ECUDA;
    const semr_summary& sm = *t.host_sum;
    if (!(sm.status & SEMR_STATUS_OVERFLOW)) {
        if (t.modes) {
            const double share = double(sm.code_total) / double(t.modes);
            if (!s->fill_seen || share > s->fill) s->fill = share;
            s->fill_seen = true;
        }
        return SEMR_OK;
    }
    // re-run once at the exact size unless the kernel also reported a device-side problem (TINY and
    // NONFINITE describe the input: they recur unchanged in the re-run)
    if (t.rerun || (sm.status & (SEMR_STATUS_TIMEOUT | SEMR_STATUS_STAGE | SEMR_STATUS_BOUNDS))) return SEMR_OK;
    semr_sizes sz;
    if (semr_sizes_for(t.mesh.lx, t.mesh.n_elem, t.fs.n_fields, t.fs.tau, &sz) != SEMR_OK) return SEMR_EINVAL;
    const uint64_t need = std::max<uint64_t>(sm.payload_bytes, sz.code_base);
    const uint64_t grow = align256(align256(need) + sz.scratch_bytes + sizeof(semr_summary) + 512 +
                                   sz.elem_report_bytes);
    if (s->budget && s->in_flight - t.bytes + grow > s->budget) return SEMR_EBUDGET;
    Ticket old = t;
    t.rerun = true;
    const int rc = ticket_launch(s, t, sz, need);
    if (rc != SEMR_OK) {
        t = old;
        t.rerun = true;
        return rc;
    }
    cudaFreeAsync(old.dev, s->stream);
    s->in_flight = s->in_flight - old.bytes + t.bytes;
    return SEMR_EAGAIN;
}

}  // namespace

extern "C" int semr_open(semr_stream** out, int device, void* cuda_stream, uint64_t mem_budget_bytes) {
    if (!out) return SEMR_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return SEMR_ECUDA;
    if (device < 0 || device >= ndev) return SEMR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return SEMR_ECUDA;
    semr_stream* s = new (std::nothrow) semr_stream;
    if (!s) return SEMR_ENOMEM;
    s->device = device;
    s->budget = mem_budget_bytes;
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return SEMR_ECUDA;
        }
        s->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return SEMR_ECUDA;
    }
    *out = s;
    return SEMR_OK;
}

extern "C" int semr_submit(semr_stream* s, const semr_fieldset* fs, const semr_mesh* mesh, uint64_t* ticket) {
    if (!s || !fs || !mesh || !ticket) return SEMR_EINVAL;
    semr_sizes sz;
    int rc = semr_sizes_for(mesh->lx, mesh->n_elem, fs->n_fields, fs->tau, &sz);
    if (rc) return rc;
    Ticket t;
    t.fs = *fs;
    t.mesh = *mesh;
    t.modes = uint64_t(fs->n_fields) * uint64_t(mesh->n_elem) * uint64_t(mesh->lx) * mesh->lx * mesh->lx;
    std::lock_guard<std::mutex> lk(s->mu);
    const double est = std::min(1.0, 2.0 * s->fill) * double(t.modes) + 4096.0;
    const uint64_t cap = std::min<uint64_t>(sz.payload_worst, sz.code_base + sz.code_width * uint64_t(est));
    const uint64_t bytes = align256(align256(cap) + sz.scratch_bytes + sizeof(semr_summary) + 512 +
                                    sz.elem_report_bytes);
    if (s->budget && s->in_flight + bytes > s->budget) return SEMR_EBUDGET;
    if (cudaSetDevice(s->device) != cudaSuccess) return SEMR_ECUDA;
    t.host_sum = pinned_get(s);
    if (!t.host_sum) return SEMR_ENOMEM;
    if (cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming) != cudaSuccess) {
        s->pinned_free.push_back(t.host_sum);
        return SEMR_ECUDA;
    }
    rc = ticket_launch(s, t, sz, cap);
    if (rc != SEMR_OK) {
        cudaEventDestroy(t.done);
        s->pinned_free.push_back(t.host_sum);
        return rc;
    }
    s->in_flight += t.bytes;
    *ticket = s->next_ticket++;
    s->tickets.emplace(*ticket, t);
    return SEMR_OK;
}

extern "C" int semr_query(semr_stream* s, uint64_t ticket) {
    if (!s) return SEMR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SEMR_EINVAL;
    if (cudaSetDevice(s->device) != cudaSuccess) return SEMR_ECUDA;
    return ticket_state(s, it->second);
}

extern "C" int semr_fetch(semr_stream* s, uint64_t ticket, int wait, void* payload, uint64_t cap,
                          uint64_t* payload_bytes, semr_field_report* reports, double* elem_report) {
    if (!s) return SEMR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SEMR_EINVAL;
    if (it->second.busy) return SEMR_EAGAIN;  // another fetch of this ticket is in progress
    if (cudaSetDevice(s->device) != cudaSuccess) return SEMR_ECUDA;
    for (;;) {  // until the results are final; waits run without the lock
        const int st = ticket_state(s, it->second);
        if (st == SEMR_OK) break;
        if (st != SEMR_EAGAIN || !wait) return st;
        const cudaEvent_t ev = it->second.done;
        it->second.busy = true;
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(ev);
        lk.lock();
        it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return SEMR_EINVAL;  // closed meanwhile
        it->second.busy = false;
        if (e != cudaSuccess) return SEMR_ECUDA;
    }
    Ticket& t = it->second;
    const semr_summary sm = *t.host_sum;
    if (payload_bytes) *payload_bytes = sm.payload_bytes;
    if (payload && cap < sm.payload_bytes) return SEMR_ENOSPACE;  // nothing copied, ticket kept
    if (reports) std::memcpy(reports, sm.field, sizeof(semr_field_report) * t.fs.n_fields);
    const uint8_t* dev = t.dev;
    const uint64_t off_elem = t.off_elem;
    const uint64_t elem_bytes = 24ull * uint64_t(t.mesh.n_elem) * t.fs.n_fields;
    const cudaEvent_t done = t.done;
    t.busy = true;
    lk.unlock();
    // copies on the stream's copy stream, ordered after the ticket's work only
    int rc = SEMR_OK;
    if (cudaStreamWaitEvent(s->copy_stream, done, 0) != cudaSuccess) rc = SEMR_ECUDA;
    if (rc == SEMR_OK && payload && sm.payload_bytes &&
        cudaMemcpyAsync(payload, dev, sm.payload_bytes, cudaMemcpyDeviceToHost, s->copy_stream) != cudaSuccess)
        rc = SEMR_ECUDA;
    if (rc == SEMR_OK && elem_report &&
        cudaMemcpyAsync(elem_report, dev + off_elem, elem_bytes, cudaMemcpyDeviceToHost, s->copy_stream) !=
            cudaSuccess)
        rc = SEMR_ECUDA;
    if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) rc = SEMR_ECUDA;
    lk.lock();
    it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SEMR_EINVAL;  // closed meanwhile
    it->second.busy = false;
    if (rc != SEMR_OK) return rc;
    release(s, it->second);
    s->tickets.erase(it);
    if (sm.status & SEMR_STATUS_TIMEOUT) return SEMR_ETIMEDOUT;
    if (sm.status & SEMR_STATUS_OVERFLOW) return SEMR_ENOSPACE;
    if (sm.status & SEMR_STATUS_NONFINITE) return SEMR_ENONFINITE;
    return SEMR_OK;
}

extern "C" void semr_close(semr_stream* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        cudaSetDevice(s->device);
        cudaStreamSynchronize(s->stream);
        cudaStreamSynchronize(s->copy_stream);
        for (auto& kv : s->tickets) release(s, kv.second);
        s->tickets.clear();
        cudaStreamSynchronize(s->stream);
        for (semr_summary* c : s->pinned_chunks) cudaFreeHost(c);
        cudaStreamDestroy(s->copy_stream);
        if (s->own_stream) cudaStreamDestroy(s->stream);
    }
    delete s;
}

// ------------------------------------------------------------ host decoder

extern "C" int semr_decode(const void* payload_v, uint64_t bytes, double* out, uint64_t cap_doubles,
                           int32_t* lx_out, int32_t* nf_out, int64_t* ne_out) {
    const uint8_t* b = static_cast<const uint8_t*>(payload_v);
    if (!b || bytes < kHeaderFixed || std::memcmp(b, "SEMR", 4) != 0) return SEMR_EINVAL;
    uint16_t version, lx, nf, flags;
    uint32_t hdr;
    uint64_t ne, code_base, code_total;
    std::memcpy(&version, b + 4, 2);
    std::memcpy(&lx, b + 6, 2);
    std::memcpy(&nf, b + 8, 2);
    std::memcpy(&flags, b + 10, 2);
    std::memcpy(&hdr, b + 12, 4);
    std::memcpy(&ne, b + 16, 8);
    std::memcpy(&code_base, b + 32, 8);
    std::memcpy(&code_total, b + 40, 8);
    if (version != kPayloadVersion || !lx_supported(lx) || nf < 1 || nf > SEMR_MAX_FIELDS) return SEMR_EINVAL;
    if (hdr != header_bytes(nf) || ne == 0 || ne >= (1ull << 40)) return SEMR_EINVAL;
    const int n3 = lx * lx * lx;
    const uint64_t mb = mask_bytes_per_elem(lx);
    const uint64_t fixed = field_fixed_bytes(lx, (int64_t)ne);
    const int width = (flags & SEMR_PAYLOAD_LOSSLESS) ? 8 : ((flags & SEMR_PAYLOAD_CODE32) ? 4 : 2);
    // (no product that can wrap: a corrupt code_total must not pass the size check)
    if (code_base != hdr + nf * fixed || code_base > bytes || code_total > (bytes - code_base) / width)
        return SEMR_EINVAL;
    if (lx_out) *lx_out = lx;
    if (nf_out) *nf_out = nf;
    if (ne_out) *ne_out = (int64_t)ne;
    if (!out) return SEMR_OK;
    if (cap_doubles < uint64_t(nf) * ne * n3) return SEMR_ENOSPACE;

    double A[SEMR_LX_MAX * SEMR_LX_MAX], Phi[SEMR_LX_MAX * SEMR_LX_MAX];
    basis_tables(lx, A, Phi, nullptr);
    std::vector<double> at(n3), t1(n3), t2(n3);
    uint64_t pos = code_base, seen_total = 0;
    for (int f = 0; f < nf; ++f) {
        const uint8_t* sec = b + hdr + f * fixed;
        const uint8_t* step = sec + pad16(ne * mb);
        const uint8_t* cnt = step + pad16(2 * ne);
        for (uint64_t e = 0; e < ne; ++e) {
            int16_t s;
            uint16_t c;
            std::memcpy(&s, step + 2 * e, 2);
            std::memcpy(&c, cnt + 2 * e, 2);
            int seen = 0;
            for (int m = 0; m < n3; ++m) {
                if (sec[e * mb + (m >> 3)] & (1u << (m & 7))) {
                    if (++seen_total > code_total) return SEMR_EINVAL;
                    if (width == 8) {
                        std::memcpy(&at[m], b + pos, 8);
                    } else if (width == 4) {
                        int32_t v;
                        std::memcpy(&v, b + pos, 4);
                        at[m] = std::ldexp((double)v, s);
                    } else {
                        int16_t v;
                        std::memcpy(&v, b + pos, 2);
                        at[m] = std::ldexp((double)v, s);
                    }
                    pos += width;
                    ++seen;
                } else {
                    at[m] = 0.0;
                }
            }
            if (seen != c) return SEMR_EINVAL;
            // u[k][j][i] = sum Phi[k][r] Phi[j][q] Phi[i][p] a[r][q][p]
            for (int r = 0; r < lx; ++r)
                for (int q = 0; q < lx; ++q)
                    for (int i = 0; i < lx; ++i) {
                        double acc = 0.0;
                        for (int pp = 0; pp < lx; ++pp) acc += Phi[i * lx + pp] * at[(r * lx + q) * lx + pp];
                        t1[(r * lx + q) * lx + i] = acc;
                    }
            for (int r = 0; r < lx; ++r)
                for (int j = 0; j < lx; ++j)
                    for (int i = 0; i < lx; ++i) {
                        double acc = 0.0;
                        for (int q = 0; q < lx; ++q) acc += Phi[j * lx + q] * t1[(r * lx + q) * lx + i];
                        t2[(r * lx + j) * lx + i] = acc;
                    }
            double* dst = out + (uint64_t(f) * ne + e) * n3;
            for (int k = 0; k < lx; ++k)
                for (int j = 0; j < lx; ++j)
                    for (int i = 0; i < lx; ++i) {
                        double acc = 0.0;
                        for (int r = 0; r < lx; ++r) acc += Phi[k * lx + r] * t2[(r * lx + j) * lx + i];
                        dst[(k * lx + j) * lx + i] = acc;
                    }
        }
    }
    return SEMR_OK;
}

extern "C" int semr_gll(int32_t lx, double* nodes, double* weights) {
    if (!lx_supported(lx)) return SEMR_EINVAL;
    return gll_nodes_weights(lx, nodes, weights);
}

extern "C" const char* semr_strerror(int code) {
    switch (code) {
        case SEMR_OK: return "ok";
        case SEMR_EINVAL: return "invalid argument";
        case SEMR_ENOMEM: return "out of memory";
        case SEMR_EBUDGET: return "request exceeds the stream's memory budget";
        case SEMR_EAGAIN: return "not finished yet";
        case SEMR_ETIMEDOUT: return "device-side wait timed out";
        case SEMR_ECUDA: return "CUDA runtime error";
        case SEMR_ENOSPACE: return "output buffer too small";
        case SEMR_ENONFINITE: return "input held NaN or infinity";
        case SEMR_EUNSUPPORTED: return "unsupported lx or precision";
        default: return "unknown status";
    }
}

extern "C" int semr_build_flags(void) {
#ifdef SEMR_BOUNDS
    return SEMR_BUILD_BOUNDS;
#else
    return 0;
#endif
}

extern "C" int semr_selftest_bounds(uint32_t* status_out) {
#ifndef SEMR_BOUNDS
    (void)status_out;
    return SEMR_EUNSUPPORTED;
#else
    if (!status_out) return SEMR_EINVAL;
    constexpr int lx = 8, n_elem = 300, n3 = lx * lx * lx;
    semr_sizes sz;
    if (semr_sizes_for(lx, n_elem, 1, 1e-3, &sz) != SEMR_OK) return SEMR_EINVAL;
    const uint64_t field_bytes = 8ull * n3 * n_elem, jac_bytes = 8ull * n_elem;
    const uint64_t total = field_bytes + jac_bytes + sz.payload_worst + sz.scratch_bytes + sizeof(semr_summary) + 1024;
    uint8_t* buf = nullptr;
    if (cudaMalloc(&buf, total) != cudaSuccess) return SEMR_ENOMEM;
    int rc = SEMR_OK;
    std::vector<double> host(static_cast<size_t>(n3) * n_elem);
    for (size_t i = 0; i < host.size(); ++i) host[i] = static_cast<double>((i * 2654435761u) % 1000u) / 1000.0 - 0.5;
    std::vector<double> jac(n_elem, 1.0);
    uint8_t* f = buf;
    uint8_t* j = f + field_bytes;
    uint8_t* pay = j + jac_bytes;
    uint8_t* scr = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(pay + sz.payload_worst) + 255) & ~uintptr_t(255));
    uint8_t* sum = scr + ((sz.scratch_bytes + 255) & ~uint64_t(255));
    if (cudaMemcpy(f, host.data(), field_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(j, jac.data(), jac_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = SEMR_ECUDA;
    } else {
        semr_fieldset fs;
        std::memset(&fs, 0, sizeof(fs));
        fs.n_fields = 1;
        fs.precision = SEMR_FP64;
        fs.tau = 1e-3;
        fs.fields[0] = reinterpret_cast<const double*>(f);
        semr_mesh mesh;
        std::memset(&mesh, 0, sizeof(mesh));
        mesh.lx = lx;
        mesh.n_elem = n_elem;
        mesh.jac = reinterpret_cast<const double*>(j);
        semr_outputs out;
        std::memset(&out, 0, sizeof(out));
        out.payload = pay;
        out.payload_cap = sz.payload_worst;
        out.summary = reinterpret_cast<semr_summary*>(sum);
        out.scratch = scr;
        out.scratch_bytes = sz.scratch_bytes;
        g_bounds_cap_short = 64;  // the fixed sections no longer fit: every element's range test fails
        rc = semr_reduce_async(&fs, &mesh, &out, nullptr);
        g_bounds_cap_short = 0;
        semr_summary h;
        if (rc == SEMR_OK && (cudaDeviceSynchronize() != cudaSuccess ||
                              cudaMemcpy(&h, sum, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess))
            rc = SEMR_ECUDA;
        if (rc == SEMR_OK) *status_out = h.status;
    }
    cudaFree(buf);
    return rc;
#endif
}
