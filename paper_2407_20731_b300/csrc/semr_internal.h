// Internal declarations shared by the CUDA path's translation units.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/semr.h"

#if defined(__CUDACC__)
#define SEMR_HD __host__ __device__
#else
#define SEMR_HD
#endif

namespace semr {

constexpr int kLxMaxTables = 16;

// Payload layout constants (format version 1; see include/semr.h).
constexpr uint16_t kPayloadVersion = 1;
constexpr uint64_t kHeaderFixed = 48;  // bytes before code_count[]

SEMR_HD inline uint64_t pad16(uint64_t b) { return (b + 15) & ~uint64_t(15); }
SEMR_HD inline uint64_t header_bytes(int n_fields) { return pad16(kHeaderFixed + 8ull * n_fields); }
SEMR_HD inline uint64_t mask_bytes_per_elem(int lx) { return (uint64_t(lx) * lx * lx + 7) / 8; }
SEMR_HD inline uint64_t field_fixed_bytes(int lx, int64_t n_elem) {
    return pad16(uint64_t(n_elem) * mask_bytes_per_elem(lx)) + 2 * pad16(2ull * uint64_t(n_elem));
}
// tau * 32767^2 > 4  <=>  2/sqrt(tau) < 32767: int16 codes suffice.
SEMR_HD inline int code_width(double tau) { return tau == 0.0 ? 8 : ((tau * 32767.0 * 32767.0 > 4.0) ? 2 : 4); }

// Host tables (semr_tables.cpp).
int gll_nodes_weights(int lx, double* x, double* w);
int basis_tables(int lx, double* A, double* Phi, double* w);

// Look-back tile state word: bits 62..63 flag, bits 0..61 value.
constexpr uint64_t kFlagAggregate = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

// Scratch layout: [control 256 B][tile_state u64 x tiles][tile_part 4 x f64 x tiles]
constexpr uint64_t kScratchControlBytes = 256;
SEMR_HD inline uint64_t scratch_bytes(uint64_t tiles) {
    return kScratchControlBytes + pad16(8 * tiles) + 32 * tiles;
}

// Warp-per-element kernel (lx = 8): look-back tiles of kWarpTile elements of one
// field, CTAs of kWarpCtaWarps warps.  Scratch: [control][tile_state][tile_part]
// [hmax_elem u32 x n_fields * n_elem][staging per resident CTA (at most
// kWarpStageCtas): for two tiles, each warp's codes in an arena of kWarpArena int16,
// the within-tile prefixes and the elements' arena offsets].  An element whose
// codes do not fit its warp's arena writes them at their final place directly.
constexpr int kWarpTile = 128;
constexpr int kWarpCtaWarps = 4;
constexpr int kWarpArena = 4096;
constexpr uint64_t kWarpStageCtas = 1024;
constexpr uint64_t kWarpStageBytes =
    (2ull * kWarpCtaWarps * kWarpArena * 2 + 2ull * (kWarpTile + 1) * 4 + 2ull * kWarpTile * 4 + 255) & ~255ull;
// The warp-group kernel (lx = 6 and 10, semr_group.cu) uses the same scratch layout with
// look-back tiles of `tile` elements (128 at lx = 6, 64 at lx = 10).
SEMR_HD inline uint64_t warp_tiles(int64_t n_elem, int32_t n_fields, int tile = kWarpTile) {
    return uint64_t(n_fields) * ((uint64_t(n_elem) + tile - 1) / tile);
}
// Bytes of the warp kernel's scratch before the staging (256-aligned).
SEMR_HD inline uint64_t warp_scratch_head(int64_t n_elem, int32_t n_fields, int tile = kWarpTile) {
    const uint64_t t = warp_tiles(n_elem, n_fields, tile);
    return (scratch_bytes(t) + pad16(4ull * uint64_t(n_fields) * uint64_t(n_elem)) + 255) & ~uint64_t(255);
}
// Full warp-kernel scratch: staging for as many CTAs as may be resident (recommended size).
SEMR_HD inline uint64_t warp_scratch_bytes(int64_t n_elem, int32_t n_fields, int tile = kWarpTile) {
    const uint64_t t = warp_tiles(n_elem, n_fields, tile);
    return warp_scratch_head(n_elem, n_fields, tile) + (t < kWarpStageCtas ? t : kWarpStageCtas) * kWarpStageBytes;
}
// Smallest usable warp-kernel scratch: staging for one CTA (a smaller scratch buffer
// limits the kernel's grid to the CTAs it can stage for).
SEMR_HD inline uint64_t warp_scratch_min(int64_t n_elem, int32_t n_fields, int tile = kWarpTile) {
    return warp_scratch_head(n_elem, n_fields, tile) + kWarpStageBytes;
}
// bytes that must be zero before each launch (control + tile states)
SEMR_HD inline uint64_t scratch_zero_bytes(uint64_t tiles) { return kScratchControlBytes + pad16(8 * tiles); }

// Elements per tile (one CTA per tile) for a given lx.
SEMR_HD constexpr int tile_elems(int lx) {
    return lx <= 2 ? 32 : lx <= 3 ? 16 : lx <= 6 ? 8 : lx <= 8 ? 4 : 2;
}

struct ScratchControl {
    uint32_t tile_counter;
    uint32_t status;
    uint32_t recomputed;  // coefficients recomputed exactly (FP64 mode)
    uint32_t done_ctas;   // warp-level kernels: CTAs finished (the last one finalizes)
};

struct LaunchParams {
    const double* fields[SEMR_MAX_FIELDS];
    double* recon[SEMR_MAX_FIELDS];
    const double* jac;
    uint8_t* payload;
    uint64_t payload_cap;
    double* elem_report;
    semr_summary* summary;
    uint8_t* scratch;
    int64_t n_elem;
    int32_t n_fields;
    int32_t tiles_per_field;
    double tau;
    int32_t lossless;
    int32_t width;
    int32_t write_recon;
    int32_t precision;
    uint64_t header_bytes;
    uint64_t fixed_bytes;
    uint64_t code_base;
    // scratch, split: control word block, look-back states, per-tile norm partials
    ScratchControl* ctl;
    uint64_t* tile_state;
    double* tile_part;
    int32_t lx;
    int32_t tile;   // elements per tile of the kernel variant that runs this item
    int32_t cumulative;  // cumulative-energy truncation (never together with lossless)
    int32_t stage_ctas;  // warp kernel: CTAs the code staging holds (its grid is at most this)
    uint32_t* hmax_elem; // warp kernel: per element-field, the largest high word of |u| (orders like max |u|)
    int16_t* code_stage; // warp kernel: kWarpTile x 512 staged codes per CTA
};

// Default scratch split of one contiguous scratch buffer.
inline void split_scratch(LaunchParams& p, uint8_t* scratch, uint64_t tiles) {
    p.scratch = scratch;
    p.ctl = reinterpret_cast<ScratchControl*>(scratch);
    p.tile_state = reinterpret_cast<uint64_t*>(scratch + kScratchControlBytes);
    p.tile_part = reinterpret_cast<double*>(scratch + kScratchControlBytes + pad16(8 * tiles));
}

// Scratch split of the warp kernel (layout of warp_scratch_bytes) for a buffer of
// `bytes` (at least warp_scratch_min): staging for as many CTAs as it holds.
inline void split_scratch_warp(LaunchParams& p, uint8_t* scratch, uint64_t bytes, int64_t n_elem, int32_t n_fields,
                               int tile = kWarpTile) {
    const uint64_t t = warp_tiles(n_elem, n_fields, tile);
    split_scratch(p, scratch, t);
    p.hmax_elem = reinterpret_cast<uint32_t*>(scratch + scratch_bytes(t));
    const uint64_t head = warp_scratch_head(n_elem, n_fields, tile);
    p.code_stage = reinterpret_cast<int16_t*>(scratch + head);
    uint64_t ctas = (bytes - head) / kWarpStageBytes;
    if (ctas > kWarpStageCtas) ctas = kWarpStageCtas;
    if (ctas > t) ctas = t;
    p.stage_ctas = (int32_t)ctas;
}

// Scratch sizes of one reduction: recommended (every kernel at full occupancy) and
// the smallest accepted (semr_api.cpp).
uint64_t scratch_need(int lx, int64_t n_elem, int32_t n_fields);
uint64_t scratch_min(int lx, int64_t n_elem, int32_t n_fields);

// Work queue of a batched launch: items of one (lx, precision) group; item i
// owns global tiles [tile_base[i], tile_base[i+1]) and fields
// [field_base[i], field_base[i+1]).
struct BatchQueue {
    const LaunchParams* items;   // device, n_items descriptors
    const uint64_t* tile_base;   // device, n_items + 1
    const uint32_t* field_base;  // device, n_items + 1
    unsigned* counter;           // device, zeroed before the launch
    int32_t n_items;
    int32_t pad_;
    uint64_t total_tiles;
    const void* tmaps;           // warp kernel: device, 64-byte aligned tensor maps, one per field (field_base order)
};

// Kernel variants (elements per tile) available for a given lx; the first is the default.
int tile_variants(int lx, int* out, int cap);
// Batched launches (semr_fast.cu / semr_kernels.cu).
int launch_reduce_fast_batch(const BatchQueue& q, int lx, int precision, int tile, void* stream);
int launch_finalize_batch(const BatchQueue& q, uint32_t total_fields, void* stream);

// Warp-per-element kernel (semr_warp.cu): lx = 8 threshold truncation in
// SEMR_FP64 / SEMR_FP32 with int16 codes.  warp_applicable() says whether it
// takes a reduction; launch_reduce_warp runs it, its last CTA finalizing (scratch
// split by split_scratch_warp, p.tile = kWarpTile).
bool warp_applicable(const LaunchParams& p);
int launch_reduce_warp(const LaunchParams& p, void* stream);
// Batched form: items of one precision and truncation (cumulative or not), each laid
// out as split_scratch_warp does except that they share one code staging (stage_ctas
// CTAs).  warp_encode_maps writes an item's n_fields tensor maps (128 bytes each) to
// host memory.
constexpr uint64_t kTensorMapBytes = 128;
int warp_encode_maps(const LaunchParams& p, void* maps);
int launch_reduce_warp_batch(const BatchQueue& q, int precision, bool cumulative, uint64_t stage_ctas, void* stream);
int launch_finalize_warp_batch(const BatchQueue& q, uint32_t total_fields, void* stream);

// Warp-group kernel (semr_group.cu): lx = 6 and 10, threshold or cumulative truncation in
// SEMR_FP64 / SEMR_FP32 with int16 codes, one element per group of one (lx = 6)
// or two (lx = 10) warps; the warp kernel's scratch layout with tiles of
// group_tile(lx) elements (0 for an lx it does not serve).
int group_tile(int lx);
bool group_applicable(const LaunchParams& p);
int launch_reduce_group(const LaunchParams& p, void* stream);
// Batched form: items of one (lx, precision, truncation), laid out as for the warp kernel (no tensor maps).
int launch_reduce_group_batch(const BatchQueue& q, int lx, int precision, bool cumulative, uint64_t stage_ctas,
                              void* stream);
int launch_finalize_group_batch(const BatchQueue& q, int lx, uint32_t total_fields, void* stream);

// Kernel launchers (semr_kernels.cu).  Return a cudaError_t value.
int launch_reduce(const LaunchParams& p, int lx, void* stream);
int launch_finalize(const LaunchParams& p, int lx, void* stream);
int launch_reduce_fast(const LaunchParams& p, int lx, void* stream);  // semr_fast.cu

}  // namespace semr
