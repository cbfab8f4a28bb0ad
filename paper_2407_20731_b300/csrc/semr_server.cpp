// Continuous-batching server for in-situ snapshot reductions.
//
// Producers (any thread) submit reductions of snapshots that already live in
// device memory (the in-situ case: the solver's fields).  A dispatcher thread
// admits queued requests in arrival order into device slots -- one CUDA
// stream each -- whenever a slot is free and the request's device memory
// (payload, scratch, reports) fits the budget next to everything admitted and
// not yet released.  Admitted requests run concurrently: their kernels
// overlap on the GPU, and a request that arrives while others are running is
// admitted as soon as a slot and memory free up.  Completion is signalled
// from the stream by a host callback, which also timestamps it; results stay
// on the device until the producer releases them.  A request's payload is
// sized for an estimate of its codes (twice the largest share of modes kept by
// the requests completed so far, 1/16 of all modes before the first, plus 4096
// codes) instead of every mode kept; a request whose codes outgrow it is re-run
// once, on its slot, at the exact size its first run reports.  This is the asynchronous
// in-situ approach of arXiv 2407.20731 (Sec. III-A: the application only
// waits for the hand-over) realised with streams inside one process.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "semr_internal.h"

using namespace semr;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    semr_fieldset fs{};
    semr_mesh mesh{};
    semr_sizes sz{};
    uint64_t bytes = 0, off_scratch = 0, off_summary = 0, off_elem = 0, payload_cap = 0, modes = 0;
    bool rerun = false;  // re-run at the exact payload size (the estimate was too small)
    double t_submit = 0, t_admit = 0, t_done = 0;
    int slot = -1;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed, 4 to be re-run at the exact size
    int status = SEMR_OK;
    uint8_t* dev = nullptr;
    semr_summary summary{};  // copied from the slot's pinned buffer when the request completes
    struct semr_server* owner = nullptr;
};

uint64_t align256(uint64_t b) { return (b + 255) & ~uint64_t(255); }

// Device block of a request for a payload of `cap` bytes: payload | scratch | summary | report.
void layout(Request* r, uint64_t cap) {
    r->payload_cap = cap;
    r->off_scratch = align256(cap);
    r->off_summary = align256(r->off_scratch + r->sz.scratch_bytes);
    r->off_elem = align256(r->off_summary + sizeof(semr_summary));
    r->bytes = align256(r->off_elem + r->sz.elem_report_bytes);
}

}  // namespace

struct semr_server {
    int device = 0;
    uint32_t slots = 1;
    uint64_t budget = 0;
    uint64_t held = 0;  // bytes of admitted, unreleased requests
    std::vector<cudaStream_t> streams;
    std::vector<int> slot_req;              // 1 busy, -1 free
    std::vector<semr_summary*> slot_summary;  // pinned, one per slot
    cudaStream_t copy_stream = nullptr;     // payload copies and frees on release
    std::mutex mu;
    std::condition_variable cv;     // dispatcher wake-up
    std::condition_variable done_cv;  // producers waiting for results
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread dispatcher;
    uint64_t admitted = 0, completed = 0;
    double busy_start = 0, busy_end = 0;
    uint64_t bytes_in_done = 0;
    double fill = 0.0;  // largest share of modes kept by a completed request
    bool fill_seen = false;
    std::deque<uint64_t> reruns;  // requests whose codes outgrew the estimate (state 4)
};

namespace {

void CUDART_CB on_done(void* arg) {
    Request* r = static_cast<Request*>(arg);
    semr_server* s = r->owner;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        std::memcpy(&r->summary, s->slot_summary[r->slot], sizeof(semr_summary));
        const uint32_t st = r->summary.status;
        if ((st & SEMR_STATUS_OVERFLOW) && !(st & (SEMR_STATUS_TIMEOUT | SEMR_STATUS_STAGE | SEMR_STATUS_BOUNDS)) &&
            !r->rerun) {
            // the codes outgrew the estimate: the dispatcher re-runs the request on its slot (which
            // stays taken) at the exact size (TINY and NONFINITE describe the input and recur
            // unchanged); no CUDA call may run in this callback
            r->state = 4;
            s->reruns.push_back(r->id);
            s->cv.notify_all();
            return;
        }
        if (r->modes && !(r->summary.status & SEMR_STATUS_OVERFLOW)) {
            const double share = double(r->summary.code_total) / double(r->modes);
            if (!s->fill_seen || share > s->fill) s->fill = share;
            s->fill_seen = true;
        }
        r->t_done = now_s();
        r->state = 2;
        s->completed += 1;
        s->busy_end = r->t_done;
        s->bytes_in_done += 8ull * r->mesh.lx * r->mesh.lx * r->mesh.lx * uint64_t(r->mesh.n_elem) * r->fs.n_fields;
        s->slot_req[r->slot] = -1;
    }
    s->cv.notify_all();
    s->done_cv.notify_all();
}

// Launch an admitted request on its slot's stream.  Called WITHOUT the lock:
// the completion callback takes the lock, and some CUDA calls wait for
// pending callbacks, so no CUDA call may run while the lock is held.
int launch(semr_server* s, Request* r) {
    cudaStream_t st = s->streams[r->slot];
    r->dev = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&r->dev), r->bytes, st) != cudaSuccess) {
        r->dev = nullptr;
        return SEMR_ENOMEM;
    }
    semr_outputs o;
    o.payload = r->dev;
    o.payload_cap = r->payload_cap;
    o.elem_report = reinterpret_cast<double*>(r->dev + r->off_elem);
    o.summary = reinterpret_cast<semr_summary*>(r->dev + r->off_summary);
    o.scratch = r->dev + r->off_scratch;
    o.scratch_bytes = r->sz.scratch_bytes;
    int rc = semr_reduce_async(&r->fs, &r->mesh, &o, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(s->slot_summary[r->slot], o.summary, sizeof(semr_summary), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return SEMR_ECUDA;
    if (cudaLaunchHostFunc(st, on_done, r) != cudaSuccess) return SEMR_ECUDA;
    return SEMR_OK;
}

// A request that could not be started (lock held on entry and exit): report it, free its slot and
// its memory (stream-ordered on the slot's stream, behind anything of it already enqueued there).
void fail_start(semr_server* s, Request* r, int rc, std::unique_lock<std::mutex>& lk) {
    uint8_t* dev = r->dev;
    cudaStream_t st = s->streams[r->slot];
    r->dev = nullptr;
    r->status = rc;
    r->state = 3;
    s->slot_req[r->slot] = -1;
    s->held -= r->bytes;
    s->done_cv.notify_all();  // r may be released (and deleted) once the lock is dropped
    if (dev) {
        lk.unlock();
        cudaFreeAsync(dev, st);
        lk.lock();
    }
}

void dispatch_loop(semr_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progressed = false;
        while (!s->reruns.empty()) {  // re-runs at the exact size, on the same slot, first
            Request* r = s->reqs[s->reruns.front()];
            const uint64_t need = std::max<uint64_t>(r->summary.payload_bytes, r->sz.code_base);
            const uint64_t old_bytes = r->bytes;
            uint8_t* old_dev = r->dev;
            Request grown = *r;
            layout(&grown, need);
            if (s->budget && s->held - old_bytes + grown.bytes > s->budget) break;  // wait for memory
            s->reruns.pop_front();
            layout(r, need);
            r->rerun = true;
            r->state = 1;
            s->held = s->held - old_bytes + r->bytes;
            lk.unlock();
            cudaFreeAsync(old_dev, s->streams[r->slot]);  // the first run is complete
            const int rc = launch(s, r);
            lk.lock();
            if (rc) fail_start(s, r, rc, lk);
            progressed = true;
        }
        while (!s->queue.empty()) {
            Request* r = s->reqs[s->queue.front()];
            int slot = -1;
            for (uint32_t k = 0; k < s->slots; ++k)
                if (s->slot_req[k] < 0) {
                    slot = (int)k;
                    break;
                }
            if (slot < 0) break;                                       // no free slot
            if (s->budget && s->held + r->bytes > s->budget) break;    // wait for memory (arrival order)
            s->queue.pop_front();
            r->slot = slot;
            r->t_admit = now_s();
            r->state = 1;
            s->slot_req[slot] = 1;
            s->held += r->bytes;
            if (s->admitted == 0) s->busy_start = r->t_admit;
            s->admitted += 1;
            lk.unlock();
            const int rc = launch(s, r);
            lk.lock();
            if (rc) fail_start(s, r, rc, lk);
            progressed = true;
        }
        if (!progressed) s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace

extern "C" int semr_server_create(semr_server** out, int device, uint32_t slots, uint64_t mem_budget_bytes) {
    if (!out || slots < 1 || slots > 64) return SEMR_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return SEMR_ECUDA;
    if (device < 0 || device >= ndev) return SEMR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return SEMR_ECUDA;
    semr_server* s = new (std::nothrow) semr_server;
    if (!s) return SEMR_ENOMEM;
    s->device = device;
    s->slots = slots;
    s->budget = mem_budget_bytes;
    s->streams.assign(slots, nullptr);
    s->slot_req.assign(slots, -1);
    s->slot_summary.assign(slots, nullptr);
    bool ok = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (uint32_t k = 0; k < slots && ok; ++k) {
        ok = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaMallocHost(&s->slot_summary[k], sizeof(semr_summary)) == cudaSuccess;
    }
    if (!ok) {
        for (uint32_t k = 0; k < slots; ++k) {
            if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
            if (s->slot_summary[k]) cudaFreeHost(s->slot_summary[k]);
        }
        if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
        delete s;
        return SEMR_ECUDA;
    }
    // keep freed request memory in the pool instead of returning it to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->dispatcher = std::thread(dispatch_loop, s);
    *out = s;
    return SEMR_OK;
}

extern "C" int semr_server_submit(semr_server* s, const semr_fieldset* fs, const semr_mesh* mesh, uint64_t* id) {
    if (!s || !fs || !mesh || !id) return SEMR_EINVAL;
    Request* r = new (std::nothrow) Request;
    if (!r) return SEMR_ENOMEM;
    int rc = semr_sizes_for(mesh->lx, mesh->n_elem, fs->n_fields, fs->tau, &r->sz);
    if (rc) {
        delete r;
        return rc;
    }
    r->fs = *fs;
    r->mesh = *mesh;
    r->modes = uint64_t(fs->n_fields) * uint64_t(mesh->n_elem) * uint64_t(mesh->lx) * mesh->lx * mesh->lx;
    double fill;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        fill = s->fill_seen ? s->fill : 1.0 / 32.0;
    }
    const double est = std::min(1.0, 2.0 * fill) * double(r->modes) + 4096.0;
    layout(r, std::min<uint64_t>(r->sz.payload_worst, r->sz.code_base + r->sz.code_width * uint64_t(est)));
    if (s->budget && r->bytes > s->budget) {
        delete r;
        return SEMR_EBUDGET;  // could never be admitted
    }
    r->owner = s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        r->t_submit = now_s();
        s->reqs[r->id] = r;
        s->queue.push_back(r->id);
        *id = r->id;
    }
    s->cv.notify_all();
    return SEMR_OK;
}

extern "C" int semr_server_wait(semr_server* s, uint64_t id, int wait, semr_request_info* info) {
    if (!s) return SEMR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return SEMR_EINVAL;
    Request* r = it->second;
    if (wait) s->done_cv.wait(lk, [&] { return r->state == 2 || r->state == 3; });
    if (r->state != 2 && r->state != 3) return SEMR_EAGAIN;  // running, queued or being re-run
    if (info) {
        info->t_submit = r->t_submit;
        info->t_admit = r->t_admit;
        info->t_done = r->t_done;
        info->slot = r->slot;
        info->status = r->status;
        info->device_bytes = r->bytes;
        if (r->state == 2) std::memcpy(&info->summary, &r->summary, sizeof(semr_summary));
    }
    if (r->state == 3) return r->status;
    const uint32_t st = r->summary.status;
    if (st & SEMR_STATUS_TIMEOUT) return SEMR_ETIMEDOUT;
    if (st & SEMR_STATUS_OVERFLOW) return SEMR_ENOSPACE;
    if (st & SEMR_STATUS_NONFINITE) return SEMR_ENONFINITE;
    return SEMR_OK;
}

extern "C" int semr_server_release(semr_server* s, uint64_t id, void* payload, uint64_t cap, uint64_t* bytes) {
    if (!s) return SEMR_EINVAL;
    Request* r = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return SEMR_EINVAL;
        r = it->second;
        s->done_cv.wait(lk, [&] { return r->state == 2 || r->state == 3; });
        s->reqs.erase(it);
    }
    // no lock held below: CUDA calls only
    int rc = SEMR_OK;
    if (r->state == 2) {
        const uint64_t n = r->summary.payload_bytes;
        if (bytes) *bytes = n;
        if (payload) {
            if (cap < n) rc = SEMR_ENOSPACE;
            else if (cudaMemcpyAsync(payload, r->dev, n, cudaMemcpyDeviceToHost, s->copy_stream) != cudaSuccess ||
                     cudaStreamSynchronize(s->copy_stream) != cudaSuccess)
                rc = SEMR_ECUDA;
        }
    }
    if (r->dev) cudaFreeAsync(r->dev, s->copy_stream);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r->state == 2) s->held -= r->bytes;
    }
    s->cv.notify_all();
    delete r;
    return rc;
}

extern "C" int semr_server_stats(semr_server* s, uint64_t* admitted, uint64_t* completed, uint64_t* queued,
                                 uint64_t* held_bytes, double* busy_seconds, uint64_t* bytes_done) {
    if (!s) return SEMR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (admitted) *admitted = s->admitted;
    if (completed) *completed = s->completed;
    if (queued) *queued = s->queue.size();
    if (held_bytes) *held_bytes = s->held;
    if (busy_seconds) *busy_seconds = s->busy_end - s->busy_start;
    if (bytes_done) *bytes_done = s->bytes_in_done;
    return SEMR_OK;
}

extern "C" void semr_server_destroy(semr_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    cudaSetDevice(s->device);
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    cudaStreamSynchronize(s->copy_stream);
    for (auto& kv : s->reqs) {
        Request* r = kv.second;
        if (r->dev) cudaFreeAsync(r->dev, s->copy_stream);
        delete r;
    }
    cudaStreamSynchronize(s->copy_stream);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (semr_summary* p : s->slot_summary) cudaFreeHost(p);
    cudaStreamDestroy(s->copy_stream);
    delete s;
}
