// Batched reduction of many snapshots in one graph-captured launch.
//
// A plan groups the snapshots by (lx, precision).  Each group runs as one
// persistent kernel whose CTAs claim tiles from a single queue that spans all
// of the group's snapshots in order (each snapshot keeps its own payload,
// look-back states and norm partials), followed by one finalize kernel over
// every (snapshot, field) of the group.  The elements per tile of each group
// are chosen by a small autotuner that times every compiled tile variant on
// the group's largest snapshot.  The whole launch sequence can be captured
// into one CUDA graph and replayed with a single graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "semr_internal.h"

using namespace semr;

namespace {

// Variants: at lx = 8, tile kWarpTile is the warp-per-element kernel; at lx = 6 and 10, tile
// group_tile(lx) is the warp-group kernel; every other tile is the CTA kernel.
struct Group {
    int lx = 0, precision = 0, tile = 0;
    bool cum = false;             // cumulative-energy truncation (warp-level kernels only)
    std::vector<int> items;       // indices into the caller's item array
    float tuned_ms[4] = {0, 0, 0, 0};
    int variants[4] = {0, 0, 0, 0};
    int n_variants = 0;
    bool warp_ok = false;         // every item fits the warp (lx = 8) or warp-group kernel
    // workspace offsets
    uint64_t off_desc = 0, off_tile_base = 0, off_field_base = 0, off_zero = 0, zero_bytes = 0;
    uint64_t off_maps = 0, off_stage = 0, stage_ctas = 0;  // warp kernel
    uint64_t total_tiles = 0;
    uint32_t total_fields = 0;
    bool warp() const { return lx == 8 && tile == kWarpTile; }               // warp-per-element kernel
    bool grp() const { return group_tile(lx) != 0 && tile == group_tile(lx); }  // warp-group kernel
    bool wl() const { return warp() || grp(); }  // either: element maxima and one shared code staging
};

// The warp-level kernel's tile of an lx (0: none).
int wl_tile(int lx) { return lx == 8 ? kWarpTile : group_tile(lx); }

uint64_t align256(uint64_t b) { return (b + 255) & ~uint64_t(255); }

int fill_params(const semr_batch_item& it, int tile, LaunchParams& p) {
    const semr_fieldset& fs = it.fs;
    const semr_mesh& m = it.mesh;
    semr_sizes sz;
    int rc = semr_sizes_for(m.lx, m.n_elem, fs.n_fields, fs.tau, &sz);
    if (rc) return rc;
    if (fs.precision != SEMR_FP64 && fs.precision != SEMR_FP32) return SEMR_EUNSUPPORTED;
    if (fs.precision == SEMR_FP64 && fs.tau == 0.0) return SEMR_EUNSUPPORTED;  // lossless FP64: single launches
    if (!m.jac || !it.out.payload || !it.out.summary) return SEMR_EINVAL;
    if (it.out.payload_cap < sz.code_base) return SEMR_EINVAL;
    const uintptr_t amask = (m.lx % 2 == 0) ? 15u : 7u;
    std::memset(&p, 0, sizeof(p));
    for (int f = 0; f < fs.n_fields; ++f) {
        if (!fs.fields[f] || (reinterpret_cast<uintptr_t>(fs.fields[f]) & amask)) return SEMR_EINVAL;
        p.fields[f] = fs.fields[f];
        p.recon[f] = (fs.flags & SEMR_WRITE_RECON) ? fs.recon[f] : nullptr;
    }
    p.jac = m.jac;
    p.payload = it.out.payload;
    p.payload_cap = it.out.payload_cap;
    p.elem_report = it.out.elem_report;
    p.summary = it.out.summary;
    p.n_elem = m.n_elem;
    p.n_fields = fs.n_fields;
    p.tiles_per_field = (int32_t)((uint64_t(m.n_elem) + tile - 1) / tile);
    p.tau = fs.tau;
    p.lossless = fs.tau == 0.0;
    p.width = (int32_t)sz.code_width;
    p.write_recon = (fs.flags & SEMR_WRITE_RECON) ? 1 : 0;
    p.precision = fs.precision;
    p.header_bytes = sz.header_bytes;
    p.fixed_bytes = field_fixed_bytes(m.lx, m.n_elem);
    p.code_base = sz.code_base;
    p.lx = m.lx;
    p.tile = tile;
    p.cumulative = (fs.flags & SEMR_CUMULATIVE) && fs.tau != 0.0 ? 1 : 0;
    return SEMR_OK;
}

uint64_t item_tiles(const semr_batch_item& it, int tile) {
    return uint64_t(it.fs.n_fields) * ((uint64_t(it.mesh.n_elem) + tile - 1) / tile);
}

}  // namespace

struct semr_batch {
    int device = 0;
    std::vector<semr_batch_item> items;
    std::vector<Group> groups;
    uint8_t* ws = nullptr;
    uint64_t ws_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Lay out the workspace for the groups' chosen tiles and upload descriptors.
int build_workspace(semr_batch* b, cudaStream_t st) {
    uint64_t off = 0;
    std::vector<std::vector<LaunchParams>> descs(b->groups.size());
    for (size_t g = 0; g < b->groups.size(); ++g) {
        Group& G = b->groups[g];
        const size_t n = G.items.size();
        G.off_desc = off;
        off = align256(off + sizeof(LaunchParams) * n);
        G.off_tile_base = off;
        off = align256(off + 8 * (n + 1));
        G.off_field_base = off;
        off = align256(off + 4 * (n + 1));
        G.total_tiles = 0;
        G.total_fields = 0;
        for (int idx : G.items) {
            G.total_tiles += item_tiles(b->items[idx], G.tile);
            G.total_fields += (uint32_t)b->items[idx].fs.n_fields;
        }
        if (G.warp()) {  // tensor maps, one per (item, field)
            G.off_maps = off;
            off = align256(off + kTensorMapBytes * G.total_fields);
        }
        G.off_zero = off;  // [counter 256][per item: control 256 + states]
        off += 256;
        for (int idx : G.items) {
            const uint64_t t = item_tiles(b->items[idx], G.tile);
            off += kScratchControlBytes + pad16(8 * t);
        }
        G.zero_bytes = off - G.off_zero;
        off = align256(off);
        for (int idx : G.items) off = align256(off + 32 * item_tiles(b->items[idx], G.tile));  // partials
        if (G.wl()) {  // per-item element maxima, then one code staging for the group
            for (int idx : G.items)
                off = align256(off + 4ull * uint64_t(b->items[idx].mesh.n_elem) * b->items[idx].fs.n_fields);
            G.stage_ctas = std::min<uint64_t>(G.total_tiles, kWarpStageCtas);
            G.off_stage = off;
            off = align256(off + G.stage_ctas * kWarpStageBytes);
        }
    }
    b->ws_bytes = std::max<uint64_t>(off, 256);
    if (cudaMalloc(reinterpret_cast<void**>(&b->ws), b->ws_bytes) != cudaSuccess) return SEMR_ENOMEM;
    // second pass: descriptors with scratch pointers into the workspace
    for (size_t g = 0; g < b->groups.size(); ++g) {
        Group& G = b->groups[g];
        const size_t n = G.items.size();
        std::vector<uint64_t> tb(n + 1, 0);
        std::vector<uint32_t> fb(n + 1, 0);
        uint64_t zoff = G.off_zero + 256;
        uint64_t poff = align256(G.off_zero + G.zero_bytes);
        uint64_t uoff = poff;  // warp-level kernels: element maxima after the partials
        if (G.wl())
            for (int idx : G.items) uoff = align256(uoff + 32 * item_tiles(b->items[idx], G.tile));
        std::vector<uint8_t> maps(G.warp() ? kTensorMapBytes * G.total_fields : 0);
        descs[g].resize(n);
        for (size_t i = 0; i < n; ++i) {
            const semr_batch_item& it = b->items[G.items[i]];
            LaunchParams& p = descs[g][i];
            int rc = fill_params(it, G.tile, p);
            if (rc) return rc;
            const uint64_t t = item_tiles(it, G.tile);
            p.scratch = b->ws + zoff;
            p.ctl = reinterpret_cast<ScratchControl*>(b->ws + zoff);
            p.tile_state = reinterpret_cast<uint64_t*>(b->ws + zoff + kScratchControlBytes);
            p.tile_part = reinterpret_cast<double*>(b->ws + poff);
            if (G.wl()) {
                p.hmax_elem = reinterpret_cast<uint32_t*>(b->ws + uoff);
                uoff = align256(uoff + 4ull * uint64_t(it.mesh.n_elem) * it.fs.n_fields);
                p.code_stage = reinterpret_cast<int16_t*>(b->ws + G.off_stage);
                p.stage_ctas = (int32_t)G.stage_ctas;
                if (G.warp() && warp_encode_maps(p, maps.data() + kTensorMapBytes * fb[i]) != 0)
                    return SEMR_EUNSUPPORTED;
            }
            zoff += kScratchControlBytes + pad16(8 * t);
            poff = align256(poff + 32 * t);
            tb[i + 1] = tb[i] + t;
            fb[i + 1] = fb[i] + (uint32_t)it.fs.n_fields;
        }
        G.total_tiles = tb[n];
        G.total_fields = fb[n];
        if (cudaMemcpyAsync(b->ws + G.off_desc, descs[g].data(), sizeof(LaunchParams) * n, cudaMemcpyHostToDevice,
                            st) != cudaSuccess ||
            cudaMemcpyAsync(b->ws + G.off_tile_base, tb.data(), 8 * (n + 1), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(b->ws + G.off_field_base, fb.data(), 4 * (n + 1), cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
            return SEMR_ECUDA;
        if (G.warp() && cudaMemcpyAsync(b->ws + G.off_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice, st) !=
                            cudaSuccess)
            return SEMR_ECUDA;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? SEMR_OK : SEMR_ECUDA;
}

BatchQueue queue_of(const semr_batch* b, const Group& G) {
    BatchQueue q{};
    q.items = reinterpret_cast<const LaunchParams*>(b->ws + G.off_desc);
    q.tile_base = reinterpret_cast<const uint64_t*>(b->ws + G.off_tile_base);
    q.field_base = reinterpret_cast<const uint32_t*>(b->ws + G.off_field_base);
    q.counter = reinterpret_cast<unsigned*>(b->ws + G.off_zero);
    q.n_items = (int32_t)G.items.size();
    q.total_tiles = G.total_tiles;
    q.tmaps = G.warp() ? b->ws + G.off_maps : nullptr;
    return q;
}

int launch_all(semr_batch* b, cudaStream_t st) {
    for (const Group& G : b->groups) {
        if (cudaMemsetAsync(b->ws + G.off_zero, 0, G.zero_bytes, st) != cudaSuccess) return SEMR_ECUDA;
        const BatchQueue q = queue_of(b, G);
        if (G.warp()) {
            if (launch_reduce_warp_batch(q, G.precision, G.cum, G.stage_ctas, st) != cudaSuccess) return SEMR_ECUDA;
            if (launch_finalize_warp_batch(q, G.total_fields, st) != cudaSuccess) return SEMR_ECUDA;
        } else if (G.grp()) {
            if (launch_reduce_group_batch(q, G.lx, G.precision, G.cum, G.stage_ctas, st) != cudaSuccess)
                return SEMR_ECUDA;
            if (launch_finalize_group_batch(q, G.lx, G.total_fields, st) != cudaSuccess) return SEMR_ECUDA;
        } else {
            if (launch_reduce_fast_batch(q, G.lx, G.precision, G.tile, st) != cudaSuccess) return SEMR_ECUDA;
            if (launch_finalize_batch(q, G.total_fields, st) != cudaSuccess) return SEMR_ECUDA;
        }
    }
    return SEMR_OK;
}

// Time the warp-level kernel of the snapshot's lx on it as a one-item batch (one
// warm-up, three timed launches); ms < 0 when it cannot run.
int probe_warp(const semr_batch_item& it, int precision, bool cum, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
               float* ms) {
    *ms = -1.0f;
    const int lx = it.mesh.lx, tile = wl_tile(lx);
    LaunchParams p;
    if (tile == 0 || fill_params(it, tile, p)) return SEMR_OK;
    const uint64_t t = item_tiles(it, tile), nf = (uint64_t)it.fs.n_fields;
    const uint64_t stage_ctas = std::min<uint64_t>(t, kWarpStageCtas);
    // [desc 1 KB][bases 512][maps][counter 256 + control + states][partials][maxima][staging]
    const uint64_t o_maps = 2048, o_zero = align256(o_maps + kTensorMapBytes * nf);
    const uint64_t zero = 256 + kScratchControlBytes + pad16(8 * t);
    const uint64_t o_part = align256(o_zero + zero), o_umax = align256(o_part + 32 * t);
    const uint64_t o_stage = align256(o_umax + 4ull * uint64_t(it.mesh.n_elem) * nf);
    const uint64_t bytes = o_stage + stage_ctas * kWarpStageBytes;
    uint8_t* w = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&w), bytes) != cudaSuccess) return SEMR_ENOMEM;
    p.scratch = w + o_zero + 256;
    p.ctl = reinterpret_cast<ScratchControl*>(w + o_zero + 256);
    p.tile_state = reinterpret_cast<uint64_t*>(w + o_zero + 256 + kScratchControlBytes);
    p.tile_part = reinterpret_cast<double*>(w + o_part);
    p.hmax_elem = reinterpret_cast<uint32_t*>(w + o_umax);
    p.code_stage = reinterpret_cast<int16_t*>(w + o_stage);
    p.stage_ctas = (int32_t)stage_ctas;
    std::vector<uint8_t> maps(kTensorMapBytes * nf);
    const uint64_t tb[2] = {0, t};
    const uint32_t fb[2] = {0, (uint32_t)nf};
    bool ok = (lx != 8 || warp_encode_maps(p, maps.data()) == 0) &&
              cudaMemcpy(w, &p, sizeof(p), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(w + 1024, tb, sizeof(tb), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(w + 1536, fb, sizeof(fb), cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(w + o_maps, maps.data(), maps.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    BatchQueue q{};
    q.items = reinterpret_cast<const LaunchParams*>(w);
    q.tile_base = reinterpret_cast<const uint64_t*>(w + 1024);
    q.field_base = reinterpret_cast<const uint32_t*>(w + 1536);
    q.counter = reinterpret_cast<unsigned*>(w + o_zero);
    q.n_items = 1;
    q.total_tiles = t;
    q.tmaps = w + o_maps;
    float total = 0.0f;
    for (int rep = 0; rep < 4 && ok; ++rep) {
        cudaMemsetAsync(w + o_zero, 0, zero, st);
        cudaEventRecord(e0, st);
        ok = (lx == 8 ? launch_reduce_warp_batch(q, precision, cum, stage_ctas, st)
                      : launch_reduce_group_batch(q, lx, precision, cum, stage_ctas, st)) == cudaSuccess;
        cudaEventRecord(e1, st);
        if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
        float m = 0.0f;
        if (ok && rep > 0 && cudaEventElapsedTime(&m, e0, e1) == cudaSuccess) total += m;
    }
    if (ok) *ms = total / 3.0f;
    else cudaGetLastError();
    cudaFree(w);
    return SEMR_OK;
}

// Time every tile variant of a group on its largest snapshot (one warm-up,
// three timed launches each) and keep the fastest.
int autotune(semr_batch* b, Group& G, cudaStream_t st) {
    int probe = G.items[0];
    for (int idx : G.items)
        if (uint64_t(b->items[idx].mesh.n_elem) * b->items[idx].fs.n_fields >
            uint64_t(b->items[probe].mesh.n_elem) * b->items[probe].fs.n_fields)
            probe = idx;
    const semr_batch_item& it = b->items[probe];
    uint64_t max_tiles = 0;
    for (int v = 0; v < G.n_variants; ++v)
        if (G.variants[v] != wl_tile(G.lx)) max_tiles = std::max(max_tiles, item_tiles(it, G.variants[v]));
    // probe workspace: descriptor, bases, counter + control + states, partials
    const uint64_t zero = 256 + kScratchControlBytes + pad16(8 * max_tiles);
    const uint64_t bytes = 4096 + zero + 32 * max_tiles + 256;
    uint8_t* w = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&w), bytes) != cudaSuccess) return SEMR_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_tile = G.variants[0];
    for (int v = 0; v < G.n_variants; ++v) {
        if (G.variants[v] == wl_tile(G.lx)) {
            float ms = -1.0f;
            const int rc = probe_warp(it, G.precision, G.cum, st, e0, e1, &ms);
            if (rc) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                cudaFree(w);
                return rc;
            }
            G.tuned_ms[v] = ms;
            if (ms >= 0.0f && ms < best) {
                best = ms;
                best_tile = G.variants[v];
            }
            continue;
        }
        LaunchParams p;
        if (fill_params(it, G.variants[v], p)) continue;
        const uint64_t t = item_tiles(it, G.variants[v]);
        uint8_t* z = w + 1024;
        p.scratch = z + 256;
        p.ctl = reinterpret_cast<ScratchControl*>(z + 256);
        p.tile_state = reinterpret_cast<uint64_t*>(z + 256 + kScratchControlBytes);
        p.tile_part = reinterpret_cast<double*>(w + 1024 + align256(zero));
        const uint64_t tb[2] = {0, t};
        const uint32_t fb[2] = {0, (uint32_t)it.fs.n_fields};
        cudaMemcpy(w, &p, sizeof(p), cudaMemcpyHostToDevice);
        cudaMemcpy(w + 512, tb, sizeof(tb), cudaMemcpyHostToDevice);
        cudaMemcpy(w + 768, fb, sizeof(fb), cudaMemcpyHostToDevice);
        BatchQueue q{};
        q.items = reinterpret_cast<const LaunchParams*>(w);
        q.tile_base = reinterpret_cast<const uint64_t*>(w + 512);
        q.field_base = reinterpret_cast<const uint32_t*>(w + 768);
        q.counter = reinterpret_cast<unsigned*>(z);
        q.n_items = 1;
        q.total_tiles = t;
        bool ok = true;
        float total = 0.0f;
        for (int rep = 0; rep < 4 && ok; ++rep) {
            cudaMemsetAsync(z, 0, 256 + kScratchControlBytes + pad16(8 * t), st);
            cudaEventRecord(e0, st);
            ok = launch_reduce_fast_batch(q, G.lx, G.precision, G.variants[v], st) == cudaSuccess;
            cudaEventRecord(e1, st);
            if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
            float ms = 0.0f;
            if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) total += ms;
        }
        if (!ok) {
            cudaGetLastError();  // a variant that does not fit this GPU is skipped
            G.tuned_ms[v] = -1.0f;
            continue;
        }
        G.tuned_ms[v] = total / 3.0f;
        if (G.tuned_ms[v] < best) {
            best = G.tuned_ms[v];
            best_tile = G.variants[v];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(w);
    G.tile = best_tile;
    return SEMR_OK;
}

}  // namespace

extern "C" int semr_batch_create(semr_batch** out, const semr_batch_item* items, int n_items, int flags,
                                 void* cuda_stream) {
    if (!out || !items || n_items < 1) return SEMR_EINVAL;
    *out = nullptr;
    semr_batch* b = new (std::nothrow) semr_batch;
    if (!b) return SEMR_ENOMEM;
    cudaGetDevice(&b->device);
    b->items.assign(items, items + n_items);
    std::map<std::tuple<int, int, bool>, int> gid;
    for (int i = 0; i < n_items; ++i) {
        LaunchParams p;
        const int rc = fill_params(items[i], tile_elems(items[i].mesh.lx), p);
        if (rc) {
            delete b;
            return rc;
        }
        const auto key = std::make_tuple(items[i].mesh.lx, items[i].fs.precision, p.cumulative != 0);
        auto f = gid.find(key);
        if (f == gid.end()) {
            Group G;
            G.lx = std::get<0>(key);
            G.precision = std::get<1>(key);
            G.cum = std::get<2>(key);
            G.n_variants = tile_variants(G.lx, G.variants, 4);
            G.tile = G.variants[0];
            gid[key] = (int)b->groups.size();
            b->groups.push_back(G);
            f = gid.find(key);
        }
        b->groups[f->second].items.push_back(i);
    }
    for (Group& G : b->groups) {  // the warp-level kernel first (the default) when every item fits it
        const int wt = wl_tile(G.lx);
        if (wt == 0) continue;
        G.warp_ok = true;
        for (int idx : G.items) {
            LaunchParams p;
            G.warp_ok = G.warp_ok && fill_params(items[idx], wt, p) == SEMR_OK &&
                        (G.lx == 8 ? warp_applicable(p) : group_applicable(p));
        }
        if (G.warp_ok) {  // first, ahead of the CTA kernel's tiles (the last of four gives way)
            const int n = std::min(G.n_variants, 3);
            for (int v = n; v > 0; --v) G.variants[v] = G.variants[v - 1];
            G.variants[0] = wt;
            G.n_variants = n + 1;
            G.tile = wt;
        }
    }
    for (Group& G : b->groups) {  // cumulative truncation: the warp-level kernels alone have a batched form
        if (!G.cum) continue;
        if (!G.warp_ok) {
            delete b;
            return SEMR_EUNSUPPORTED;
        }
        G.variants[0] = G.tile = wl_tile(G.lx);
        G.n_variants = 1;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (flags & SEMR_BATCH_AUTOTUNE) {
        for (Group& G : b->groups) {
            if (G.n_variants > 1) {
                const int rc = autotune(b, G, st);
                if (rc) {
                    delete b;
                    return rc;
                }
            }
        }
    }
    const int rc = build_workspace(b, st);
    if (rc) {
        if (b->ws) cudaFree(b->ws);
        delete b;
        return rc;
    }
    *out = b;
    return SEMR_OK;
}

extern "C" int semr_batch_launch(semr_batch* b, void* cuda_stream) {
    if (!b) return SEMR_EINVAL;
    return launch_all(b, static_cast<cudaStream_t>(cuda_stream));
}

extern "C" int semr_batch_capture(semr_batch* b, void* cuda_stream) {
    if (!b) return SEMR_EINVAL;
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return SEMR_ECUDA;
    int rc = SEMR_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = SEMR_ECUDA;
    if (rc == SEMR_OK) {
        rc = launch_all(b, cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (rc == SEMR_OK && e != cudaSuccess) rc = SEMR_ECUDA;
        if (rc == SEMR_OK) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            b->exec = nullptr;
            b->graph = g;
            if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
                b->exec = nullptr;  // replay refuses (SEMR_EINVAL) until a capture succeeds
                rc = SEMR_ECUDA;
            }
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    cudaStreamDestroy(cap);
    (void)cuda_stream;
    return rc;
}

extern "C" int semr_batch_replay(semr_batch* b, void* cuda_stream) {
    if (!b || !b->exec) return SEMR_EINVAL;
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? SEMR_OK : SEMR_ECUDA;
}

extern "C" int semr_batch_schedule(const semr_batch* b, int group, int* lx, int* precision, int* tile,
                                   int* n_items, float* variant_ms, int* variant_tiles, int cap) {
    if (!b) return SEMR_EINVAL;
    if (group < 0) return (int)b->groups.size();  // number of groups
    if (group >= (int)b->groups.size()) return SEMR_EINVAL;
    const Group& G = b->groups[group];
    if (lx) *lx = G.lx;
    if (precision) *precision = G.precision;
    if (tile) *tile = G.tile;
    if (n_items) *n_items = (int)G.items.size();
    for (int v = 0; v < G.n_variants && v < cap; ++v) {
        if (variant_ms) variant_ms[v] = G.tuned_ms[v];
        if (variant_tiles) variant_tiles[v] = G.variants[v];
    }
    return SEMR_OK;
}

extern "C" void semr_batch_destroy(semr_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ws) cudaFree(b->ws);
    delete b;
}
