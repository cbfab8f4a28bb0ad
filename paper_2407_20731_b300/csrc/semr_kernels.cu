// Fused reduce kernel and finalize kernel of the in-situ SEM snapshot
// reduction (arXiv 2407.20731, Sec. IV-B: JPEG-like spectral truncation of
// spectral-element fields, keeping the most energetic modes under an allowed
// error; Eq. 1 for the compression ratio).
//
// One CTA reduces one tile of TILE consecutive elements of one field.  Each
// element block of lx^3 values is owned by lx^2 threads, one per "pencil"
// (a line of lx values); the three small dense contractions of each
// transform run in registers along the pencil, with two padded shared-memory
// transposes between directions.  The pencil a thread holds after the
// inverse transform is the one it loaded, so the input block stays in
// registers for the error norms and is read from HBM exactly once.
//
// Per tile:  load u (FP64, vectorised)  ->  forward transform (even-odd
// folded)  ->  S_e = sum a^2 (FP64)  ->  threshold, step exponent  ->  mask
// bits (shared atomics), word prefix popcounts  ->  tile aggregate published
// for the decoupled look-back  ->  quantise, stage codes in shared memory
// ->  inverse transform  ->  error partials, segmented reductions  ->
// look-back for the tile's global code offset  ->  coalesced writes of
// masks, steps, counts, codes, element report, tile partials.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "semr_device.cuh"

namespace semr {

// ------------------------------------------------------------ tables

template <int LX, typename T>
struct Tables {
    T A[LX * LX];    // analysis  A[p*LX + i] = phi_p(x_i) w_i
    T Phi[LX * LX];  // synthesis Phi[i*LX + p] = phi_p(x_i)
    double w[LX];    // GLL weights (norms are always FP64)
};

// -------------------------------------------------- kernel configuration

template <int LX>
struct Cfg {
    static constexpr int NP = LX * LX;             // pencils (threads) per element
    static constexpr int N3 = LX * LX * LX;        // values per element
    static constexpr int TILE = tile_elems(LX);    // elements per CTA
    static constexpr int NT = TILE * NP;           // active threads
    static constexpr int BLOCK = (NT + 31) / 32 * 32;
    static constexpr int NW = BLOCK / 32;
    static constexpr int MW = (N3 + 31) / 32;      // 32-bit mask words per element
    static constexpr int SY = LX + 1;              // padded transpose strides
    static constexpr int SX = LX * (LX + 1);
    static constexpr int BUFN = LX * SX;           // padded block size (elements of T)
};

template <int LX, typename T>
struct Smem {
    using C = Cfg<LX>;
    static constexpr size_t buf_bytes = sizeof(T) * C::TILE * C::BUFN;
    static constexpr size_t off_buf0 = 0;
    static constexpr size_t off_buf1 = off_buf0 + buf_bytes;
    static constexpr size_t off_codes = off_buf1 + buf_bytes;                 // 8 B per code max
    static constexpr size_t off_red = off_codes + 8ull * C::TILE * C::N3;     // 4 x BLOCK doubles
    static constexpr size_t off_elem = off_red + 32ull * C::BLOCK;            // TILE x 8 doubles
    static constexpr size_t off_mask = off_elem + 64ull * C::TILE;            // TILE x MW u32
    static constexpr size_t off_wpre = off_mask + 4ull * C::TILE * C::MW;     // TILE x MW u32
    static constexpr size_t off_misc = off_wpre + 4ull * C::TILE * C::MW;     // ints
    static constexpr size_t bytes = off_misc + 4ull * (4 * C::TILE + 16);
};

// Segmented reduction over the NP threads of each element of the tile:
// (sum v0, sum v1, max v2, max v3) -> out[lt*8 + 0..3].  Deterministic order.
template <int LX>
__device__ __forceinline__ void seg_reduce4(double* red, double* out, double v0, double v1, double v2,
                                            double v3) {
    using C = Cfg<LX>;
    const int tid = threadIdx.x;
    red[tid] = v0;
    red[C::BLOCK + tid] = v1;
    red[2 * C::BLOCK + tid] = v2;
    red[3 * C::BLOCK + tid] = v3;
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (int lt = warp; lt < C::TILE; lt += C::NW) {
        double s0 = 0.0, s1 = 0.0, m2 = 0.0, m3 = 0.0;
        for (int i = lane; i < C::NP; i += 32) {
            const int k = lt * C::NP + i;
            s0 += red[k];
            s1 += red[C::BLOCK + k];
            m2 = fmax(m2, red[2 * C::BLOCK + k]);
            m3 = fmax(m3, red[3 * C::BLOCK + k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
            m3 = fmax(m3, __shfl_xor_sync(0xffffffffu, m3, o));
        }
        if (lane == 0) {
            out[lt * 8 + 0] = s0;
            out[lt * 8 + 1] = s1;
            out[lt * 8 + 2] = m2;
            out[lt * 8 + 3] = m3;
        }
    }
    __syncthreads();
}

// ------------------------------------------------------------ the kernel

template <int LX, typename T>
__global__ void __launch_bounds__(Cfg<LX>::BLOCK)
reduce_kernel(const LaunchParams p, const Tables<LX, T> tab) {
    using C = Cfg<LX>;
    using S = Smem<LX, T>;
    constexpr int NP = C::NP, N3 = C::N3, TILE = C::TILE, MW = C::MW;
    constexpr int SX = C::SX, SY = C::SY;
    extern __shared__ __align__(16) uint8_t smem[];
    T* buf0 = reinterpret_cast<T*>(smem + S::off_buf0);
    T* buf1 = reinterpret_cast<T*>(smem + S::off_buf1);
    uint8_t* scodes = smem + S::off_codes;
    double* red = reinterpret_cast<double*>(smem + S::off_red);
    double* selem = reinterpret_cast<double*>(smem + S::off_elem);  // [TILE][8]
    uint32_t* smask = reinterpret_cast<uint32_t*>(smem + S::off_mask);
    uint32_t* swpre = reinterpret_cast<uint32_t*>(smem + S::off_wpre);
    int* smisc = reinterpret_cast<int*>(smem + S::off_misc);
    int* s_cnt = smisc;                 // [TILE]
    int* s_epre = smisc + TILE;         // [TILE+1]
    int* s_step = smisc + 2 * TILE + 1; // [TILE]
    unsigned long long* s_tile = reinterpret_cast<unsigned long long*>(smisc + 4 * TILE + 2);

    ScratchControl* ctl = p.ctl;
    uint64_t* tile_state = p.tile_state;
    const uint64_t n_tiles = (uint64_t)p.n_fields * p.tiles_per_field;
    double* tile_part = p.tile_part;

    const int tid = threadIdx.x;
    if (tid == 0) s_tile[0] = atomicAdd(&ctl->tile_counter, 1u);
    for (int i = tid; i < TILE * MW; i += C::BLOCK) smask[i] = 0u;
    __syncthreads();
    const uint64_t tile = s_tile[0];
    if (tile >= n_tiles) return;  // uniform across the CTA
    const int f = (int)(tile / p.tiles_per_field);
    const int64_t e0 = (int64_t)(tile % p.tiles_per_field) * TILE;
    const int n_here = (p.n_elem - e0 < TILE) ? (int)(p.n_elem - e0) : TILE;
    // bounds build: the tile's elements and its field's section of the payload (every write of
    // the tile below is skipped if they fall outside their buffers)
    const bool tok = bchk(f < p.n_fields && n_here >= 1 &&
                              pad16((uint64_t)p.n_elem * ((N3 + 7) / 8)) + 2 * pad16(2ull * p.n_elem) <= p.fixed_bytes &&
                              p.header_bytes + (f + 1ull) * p.fixed_bytes <= p.code_base &&
                              p.code_base <= p.payload_cap,
                          &p.ctl->status);

    const int lt = tid / NP;    // element within the tile
    const int P = tid % NP;     // pencil index
    const int pa = P / LX, pb = P % LX;
    const bool active = (tid < C::NT) && (lt < n_here);
    const int64_t e = e0 + lt;
    T* b0 = buf0 + (lt < TILE ? lt : 0) * C::BUFN;
    T* b1 = buf1 + (lt < TILE ? lt : 0) * C::BUFN;

    // ---- load the pencil u[k=pa][j=pb][0..LX-1]
    double u[LX];
    if (active) {
        const double* src = p.fields[f] + e * N3 + P * LX;
        if constexpr ((LX % 2) == 0) {
#pragma unroll
            for (int i = 0; i < LX; i += 2) {
                double2 v = __ldg(reinterpret_cast<const double2*>(src + i));
                u[i] = v.x;
                u[i + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < LX; ++i) u[i] = __ldg(src + i);
        }
    } else {
#pragma unroll
        for (int i = 0; i < LX; ++i) u[i] = 0.0;
    }

    // ---- forward transform: along i (registers), j, k (via shared memory)
    T x[LX], y[LX];
#pragma unroll
    for (int i = 0; i < LX; ++i) x[i] = (T)u[i];
    fwd1d<LX, T>(tab.A, x, y);  // y = t1[k][j][p], p = 0..LX-1
    if (lt < TILE) {
#pragma unroll
        for (int q = 0; q < LX; ++q) b0[pa * SX + pb * SY + q] = y[q];  // [k][j][p]
    }
    __syncthreads();
    if (lt < TILE) {  // thread (k = pa, p = pb) reads t1[k][0..][p]
#pragma unroll
        for (int j = 0; j < LX; ++j) x[j] = b0[pa * SX + j * SY + pb];
    }
    fwd1d<LX, T>(tab.A, x, y);  // y = t2[k][q][p], q = 0..LX-1
    if (lt < TILE) {
#pragma unroll
        for (int q = 0; q < LX; ++q) b1[pa * SX + q * SY + pb] = y[q];  // [k][q][p]
    }
    __syncthreads();
    if (lt < TILE) {  // thread (q = pa, p = pb) reads t2[0..][q][p]
#pragma unroll
        for (int k = 0; k < LX; ++k) x[k] = b1[k * SX + pa * SY + pb];
    }
    T a[LX];
    fwd1d<LX, T>(tab.A, x, a);  // a[r] = a[r][q=pa][p=pb], mode m = P + NP*r

    // ---- element energy S_e = sum_m a_m^2 in FP64
    double spart = 0.0;
#pragma unroll
    for (int r = 0; r < LX; ++r) spart = fma((double)a[r], (double)a[r], spart);
    if (!active) spart = 0.0;
    seg_reduce4<LX>(red, selem, spart, 0.0, 0.0, 0.0);

    // ---- per element: threshold t, step s_e, magnitude threshold g (one thread each)
    if (tid < TILE) {
        const int l = tid;
        const double Se = selem[l * 8 + 0];
        int step = INT16_MIN, mode = 0;  // mode 0: keep none, 1: threshold, 2: keep all (lossless)
        double g64 = 0.0;
        if (l < n_here) {
            if (!isfinite(Se)) {
                atomicOr(&ctl->status, (unsigned)SEMR_STATUS_NONFINITE);
            } else if (p.lossless) {
                mode = 2;
            } else {
                const double t = p.tau * Se;
                if (t >= DBL_MIN && isfinite(t)) {
                    const long long bits = __double_as_longlong(t);
                    const int ex = (int)((bits >> 52) & 0x7ff) - 1022;  // t = mu 2^ex, mu in [1/2,1)
                    step = (ex - 1) >> 1;                               // floor((ex-1)/2)
                    mode = 1;
                    if constexpr (sizeof(T) == 8) g64 = threshold_abs64(t);
                    else g64 = (double)threshold_abs32(t);
                } else if (!isfinite(t)) {
                    atomicOr(&ctl->status, (unsigned)SEMR_STATUS_NONFINITE);
                }
            }
        }
        selem[l * 8 + 4] = g64;
        s_step[l] = step;
        reinterpret_cast<int*>(&selem[l * 8 + 5])[0] = mode;
    }
    __syncthreads();

    const int emode = (lt < TILE) ? reinterpret_cast<const int*>(&selem[lt * 8 + 5])[0] : 0;
    const int step = (lt < TILE) ? s_step[lt] : 0;
    const T g = (lt < TILE) ? (T)selem[lt * 8 + 4] : (T)0;

    // ---- mask bits
    bool keep[LX];
#pragma unroll
    for (int r = 0; r < LX; ++r) {
        keep[r] = active && (emode == 2 || (emode == 1 && fabs(a[r]) >= g));
        if (keep[r]) {
            const int m = P + NP * r;
            atomicOr(&smask[lt * MW + (m >> 5)], 1u << (m & 31));
        }
    }
    __syncthreads();
    // word prefix popcounts and counts, one warp per element
    {
        const int warp = tid >> 5, lane = tid & 31;
        for (int l = warp; l < TILE; l += C::NW) {
            uint32_t carry = 0;
            for (int w0 = 0; w0 < MW; w0 += 32) {
                const int w = w0 + lane;
                const uint32_t c = (w < MW) ? __popc(smask[l * MW + w]) : 0u;
                uint32_t incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                if (w < MW) swpre[l * MW + w] = carry + incl - c;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) s_cnt[l] = (int)carry;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int l = 0; l < TILE; ++l) {
            s_epre[l] = acc;
            acc += (l < n_here) ? s_cnt[l] : 0;
        }
        s_epre[TILE] = acc;
        // publish the tile aggregate for the look-back
        const uint64_t v = (uint64_t)acc & kValueMask;
        if (tok) st_release_u64(&tile_state[tile], (tile == 0 ? kFlagPrefix : kFlagAggregate) | v);
    }
    __syncthreads();

    // ---- quantise kept modes, stage codes in shared memory (tile order)
    const int width = p.width;
    T at[LX];
#pragma unroll
    for (int r = 0; r < LX; ++r) {
        at[r] = (T)0;
        if (keep[r]) {
            const int m = P + NP * r;
            const uint32_t wm = smask[lt * MW + (m >> 5)];
            const int rank = (int)swpre[lt * MW + (m >> 5)] + __popc(wm & ((1u << (m & 31)) - 1u));
            const int pos = s_epre[lt] + rank;
            if (emode == 2) {
                reinterpret_cast<double*>(scodes)[pos] = (double)a[r];
                at[r] = a[r];
            } else {
                long long c;
                if constexpr (sizeof(T) == 8) {
                    const double cd = rint(a[r] * pow2d(-step));
                    c = (long long)cd;
                    at[r] = cd * pow2d(step);
                } else {
                    if (step >= -126 && step <= 127) {
                        const float cf = rintf(a[r] * pow2f(-step));
                        c = (long long)cf;
                        at[r] = cf * pow2f(step);
                    } else {
                        const double cd = rint((double)a[r] * pow2d(-step));
                        c = (long long)cd;
                        at[r] = (T)(cd * pow2d(step));
                    }
                }
                if (width == 2) reinterpret_cast<int16_t*>(scodes)[pos] = (int16_t)c;
                else reinterpret_cast<int32_t*>(scodes)[pos] = (int32_t)c;
            }
        }
    }

    // ---- inverse transform: along r (registers), q, p (via shared memory)
    inv1d<LX, T>(tab.Phi, at, y);  // y[k] = v[k][q=pa][p=pb]
    if (lt < TILE) {
#pragma unroll
        for (int k = 0; k < LX; ++k) b0[k * SX + pa * SY + pb] = y[k];  // [k][q][p]
    }
    __syncthreads();
    if (lt < TILE) {  // thread (k = pa, p = pb) reads v[k][0..][p]
#pragma unroll
        for (int q = 0; q < LX; ++q) x[q] = b0[pa * SX + q * SY + pb];
    }
    inv1d<LX, T>(tab.Phi, x, y);  // y[j] = v2[k][j][p]
    if (lt < TILE) {
#pragma unroll
        for (int j = 0; j < LX; ++j) b1[pa * SX + j * SY + pb] = y[j];  // [k][j][p]
    }
    __syncthreads();
    if (lt < TILE) {  // thread (k = pa, j = pb) reads v2[k][j][0..]
#pragma unroll
        for (int q = 0; q < LX; ++q) x[q] = b1[pa * SX + pb * SY + q];
    }
    inv1d<LX, T>(tab.Phi, x, y);  // y[i] = u~[k][j][i]

    // ---- error partials (FP64)
    double e2p = 0.0, enp = 0.0, linf = 0.0, umax = 0.0;
    if (active) {
        const double wjk = tab.w[pa] * tab.w[pb];
#pragma unroll
        for (int i = 0; i < LX; ++i) {
            const double d = u[i] - (double)y[i];
            const double wq = tab.w[i] * wjk;
            e2p = fma(wq * d, d, e2p);
            enp = fma(wq * u[i], u[i], enp);
            linf = fmax(linf, fabs(d));
            umax = fmax(umax, fabs(u[i]));
        }
        if (p.write_recon && p.recon[f] && tok) {
            double* dst = p.recon[f] + e * N3 + P * LX;
#pragma unroll
            for (int i = 0; i < LX; ++i) dst[i] = (double)y[i];
        }
    }
    seg_reduce4<LX>(red, selem, e2p, enp, linf, umax);  // selem[l*8 + 0..3]

    // ---- look-back for the tile's code offset
    if (tid == 0) {
        const uint64_t agg = (uint64_t)s_epre[TILE];
        uint64_t excl = 0;
        if (tile > 0) {
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const uint64_t v = ld_acquire_u64(&tile_state[j]);
                const uint64_t flag = v & ~kValueMask;
                if (flag == kFlagPrefix) {
                    excl += v & kValueMask;
                    break;
                } else if (flag == kFlagAggregate) {
                    excl += v & kValueMask;
                    --j;
                } else {
                    if (++spins > (1u << 22)) {
                        atomicOr(&ctl->status, (unsigned)SEMR_STATUS_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (tok) st_release_u64(&tile_state[tile], kFlagPrefix | ((excl + agg) & kValueMask));
        }
        s_tile[1] = excl;
        // per-tile partials for the field reductions
        double s0 = 0.0, s1 = 0.0, m2 = 0.0, m3 = 0.0;
        for (int l = 0; l < n_here; ++l) {
            const double J = p.jac[e0 + l];
            s0 += J * selem[l * 8 + 0];
            s1 += J * selem[l * 8 + 1];
            m2 = fmax(m2, selem[l * 8 + 2]);
            m3 = fmax(m3, selem[l * 8 + 3]);
        }
        if (tok) {
            double* tp = tile_part + 4 * tile;
            tp[0] = s0;
            tp[1] = s1;
            tp[2] = m2;
            tp[3] = m3;
        }
    }
    __syncthreads();
    const uint64_t tile_excl = s_tile[1];

    // ---- writes: codes (contiguous for the tile), masks, steps, counts, element report
    {
        const uint64_t ncodes = (uint64_t)s_epre[TILE];
        const uint64_t gbyte = p.code_base + (uint64_t)width * tile_excl;
        const uint64_t nbytes = (uint64_t)width * ncodes;
        if (!tok) {
            // (bounds build) nothing of this tile is written
        } else if (gbyte + nbytes <= p.payload_cap) {
            uint8_t* dst = p.payload + gbyte;
            if (width == 8) {  // 8-byte aligned: code_base is 16-aligned
                const double* sc = reinterpret_cast<const double*>(scodes);
                for (uint64_t i = tid; i < ncodes; i += C::BLOCK) reinterpret_cast<double*>(dst)[i] = sc[i];
            } else if (width == 4) {
                const int32_t* sc = reinterpret_cast<const int32_t*>(scodes);
                for (uint64_t i = tid; i < ncodes; i += C::BLOCK) reinterpret_cast<int32_t*>(dst)[i] = sc[i];
            } else {
                const int16_t* sc = reinterpret_cast<const int16_t*>(scodes);
                for (uint64_t i = tid; i < ncodes; i += C::BLOCK) reinterpret_cast<int16_t*>(dst)[i] = sc[i];
            }
        } else if (tid == 0 && nbytes > 0) {
            atomicOr(&ctl->status, (unsigned)SEMR_STATUS_OVERFLOW);
        }
    }
    if (tok) {
        constexpr int mb = (N3 + 7) / 8;
        uint8_t* fsec = p.payload + p.header_bytes + (uint64_t)f * p.fixed_bytes;
        uint8_t* mdst = fsec + (uint64_t)e0 * mb;
        const uint8_t* msrc = reinterpret_cast<const uint8_t*>(smask);
        for (int i = tid; i < n_here * mb; i += C::BLOCK) {
            const int l = i / mb, b = i % mb;
            mdst[i] = msrc[l * MW * 4 + b];
        }
        int16_t* sdst = reinterpret_cast<int16_t*>(fsec + pad16((uint64_t)p.n_elem * mb));
        uint16_t* cdst = reinterpret_cast<uint16_t*>(fsec + pad16((uint64_t)p.n_elem * mb) + pad16(2ull * p.n_elem));
        if (tid < n_here) {
            sdst[e0 + tid] = (int16_t)s_step[tid];
            cdst[e0 + tid] = (uint16_t)s_cnt[tid];
        }
        // the field's last tile zeroes the 16-byte padding after each section
        if (e0 + n_here == p.n_elem && tid < 16) {
            const uint64_t me = (uint64_t)p.n_elem * mb;
            if (me + tid < pad16(me)) fsec[me + tid] = 0;
            const uint64_t se = 2ull * p.n_elem;
            uint8_t* sb = reinterpret_cast<uint8_t*>(sdst);
            uint8_t* cb = reinterpret_cast<uint8_t*>(cdst);
            if (se + tid < pad16(se)) {
                sb[se + tid] = 0;
                cb[se + tid] = 0;
            }
        }
        if (p.elem_report && tid < 3 * n_here) {
            const int l = tid / 3, c = tid % 3;
            double v = selem[l * 8 + c];
            if (c < 2) v *= p.jac[e0 + l];
            p.elem_report[((uint64_t)f * p.n_elem + e0) * 3 + tid] = v;
        }
    }
}

// ------------------------------------------------------ finalize kernel

__global__ void __launch_bounds__(256) finalize_kernel(const LaunchParams p, int lx) {
    __shared__ double red[4][256];
    finalize_field(p, blockIdx.x, lx, red, p.tile_part, (uint64_t)p.tiles_per_field);
}

// One block per (item, field) of a batched launch.
__global__ void __launch_bounds__(256) finalize_batch_kernel(const BatchQueue q) {
    __shared__ double red[4][256];
    __shared__ int s_item;
    if (threadIdx.x == 0) {
        int lo = 0, hi = q.n_items - 1;  // last item with field_base <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (q.field_base[mid] <= blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_item = lo;
    }
    __syncthreads();
    const LaunchParams& p = q.items[s_item];
    finalize_field(p, (int)(blockIdx.x - q.field_base[s_item]), p.lx, red, p.tile_part, (uint64_t)p.tiles_per_field);
}

// ------------------------------------------------------------ launchers

namespace {

template <int LX, typename T>
int launch_lx(const LaunchParams& p, void* stream) {
    using C = Cfg<LX>;
    Tables<LX, T> tab;
    double A[LX * LX], Phi[LX * LX], w[LX];
    int rc = basis_tables(LX, A, Phi, w);
    if (rc) return (int)cudaErrorInvalidValue;
    for (int i = 0; i < LX * LX; ++i) {
        tab.A[i] = (T)A[i];
        tab.Phi[i] = (T)Phi[i];
    }
    for (int i = 0; i < LX; ++i) tab.w[i] = w[i];
    const size_t smem = Smem<LX, T>::bytes;
    cudaError_t err = cudaFuncSetAttribute(reduce_kernel<LX, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return (int)err;
    const uint64_t tiles = (uint64_t)p.n_fields * p.tiles_per_field;
    reduce_kernel<LX, T><<<(unsigned)tiles, C::BLOCK, smem, (cudaStream_t)stream>>>(p, tab);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_dispatch(const LaunchParams& p, int lx, void* stream) {
    switch (lx) {
        case 2: return launch_lx<2, T>(p, stream);
        case 3: return launch_lx<3, T>(p, stream);
        case 4: return launch_lx<4, T>(p, stream);
        case 5: return launch_lx<5, T>(p, stream);
        case 6: return launch_lx<6, T>(p, stream);
        case 7: return launch_lx<7, T>(p, stream);
        case 8: return launch_lx<8, T>(p, stream);
        case 9: return launch_lx<9, T>(p, stream);
        case 10: return launch_lx<10, T>(p, stream);
        case 11: return launch_lx<11, T>(p, stream);
        case 12: return launch_lx<12, T>(p, stream);
        default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace

int launch_reduce(const LaunchParams& p, int lx, void* stream) {
    // lossless FP64 stores every coefficient as an FP64 value: hardware FP64 path
    if (p.precision == SEMR_FP64_NATIVE || (p.precision == SEMR_FP64 && p.lossless))
        return launch_dispatch<double>(p, lx, stream);
    return launch_reduce_fast(p, lx, stream);
}

int launch_finalize(const LaunchParams& p, int lx, void* stream) {
    finalize_kernel<<<p.n_fields, 256, 0, (cudaStream_t)stream>>>(p, lx);
    return (int)cudaGetLastError();
}

int launch_finalize_batch(const BatchQueue& q, uint32_t total_fields, void* stream) {
    finalize_batch_kernel<<<total_fields, 256, 0, (cudaStream_t)stream>>>(q);
    return (int)cudaGetLastError();
}

}  // namespace semr
