// In-situ slice image (arXiv 2407.20731, Sec. IV-A: images of a slice through
// the turbulent fields, generated while the simulation runs).  The image is a
// headless RGBA8 device buffer; the steps are those stated in semr.h:
// pixel centres and element ownership in FP64 (they decide which element
// owns a pixel, bit for bit as a plain FP64 evaluation), interpolation and
// colour in FP32 (B300's FP32 pipes run ~50x its FP64 pipe, and 8-bit colour
// needs ~1e-3 relative accuracy).
//
// Axis-aligned slices (the usual case: a plane normal to x, y or z, image
// axes along the other two) run one thread block per element of the sliced
// layer: the block loads the element once, contracts it along the slice
// normal with l_t(zeta) (lx^3 FMAs per component), then every pixel it owns
// costs lx^2 + lx FMAs per component from shared memory.  A pixel's column
// depends only on the column index and its row only on the row index, so
// the pixels an element owns form a rectangle, found exactly by testing a
// window of candidate columns and rows with the FP64 ownership rule.  Any
// other plane takes the per-pixel path (lx^3 FMAs, element values through the
// read-only cache).
#include <climits>
#include <cmath>
#include <cstring>

#include "semr_device.cuh"

namespace semr {
namespace {

constexpr int kMaxCtrl = SEMR_SLICE_MAX_CTRL;
constexpr int kMaxComp = SEMR_SLICE_MAX_COMP;
constexpr int kChunk = 64;        // columns (rows) whose basis values one block holds at a time
constexpr int kAxisThreads = 128;  // threads of an element's block
constexpr int kWinCache = 256;     // candidate-window entries whose reference coordinate is kept

struct SliceArgs {
    const double* f[kMaxComp];
    uint8_t* rgba;
    float* values;
    int32_t lx, nc;
    int32_t n[3];
    double mo[3], h[3];
    double o[3], U[3], V[3];
    int32_t W, H;
    float vmin, inv_range;
    int32_t n_ctrl;
    float ct[kMaxCtrl], cinvw[kMaxCtrl], cr[kMaxCtrl], cg[kMaxCtrl], cb[kMaxCtrl];
    float dr[kMaxCtrl], dg[kMaxCtrl], db[kMaxCtrl];  // channel steps of each segment
    uint32_t bg;
    float xn[SEMR_LX_MAX];  // GLL nodes
    float lw[SEMR_LX_MAX];  // 1 / prod_{m != i} (x_i - x_m)
    // axis-aligned path
    int32_t ax_a, ax_b, ax_n;  // lattice axis of the columns, of the rows, of the normal
    int32_t layer;             // element index along the normal (-1: the plane misses the lattice)
    float Ln[SEMR_LX_MAX];     // l_t(zeta) along the normal
    int32_t ea0, eb0, na, nb;  // element range of the layer covered by the grid
    // fast ownership test: reciprocals and, per axis, the distance to an integer
    // below which q is recomputed with correctly rounded operations
    double inv_W, inv_H, inv_h[3], near_int[3];
    double px_per[2];  // axis path: pixels per unit length along the column and the row axis
    // axis path, per side (0: columns, 1: rows): q(c) = A + (c + 0.5) B as floats
    // with the distance to an integer below which the exact rule decides, and
    // in FP64 for the reference coordinate
    float Af[2], Bf[2], thr_f[2];
    double Ad[2], Bd[2];
};

__device__ __forceinline__ double frac_of(int i, int n) { return __ddiv_rn((double)i + 0.5, (double)n); }

// Steps 1-2 along lattice axis `ax` for pixel column c and row r: element
// index along the axis (-1 outside) and reference coordinate.  The element
// index is exactly floor(q) of the correctly rounded evaluation (every
// operation rounded once, no contraction into FMAs): q is first formed with
// multiplications by reciprocals (error far below near_int), and only when it
// lies within near_int of an integer, where the floor could differ, is it
// recomputed with correctly rounded divisions (B300 runs FP64 division on its
// slow FP64 pipe).  xi feeds the FP32 basis only, so the fast q serves it.
__device__ __forceinline__ int locate_axis(const SliceArgs& a, int ax, int c, int r, double& xi) {
    double q = (fma((double)c + 0.5, a.inv_W * a.U[ax], a.o[ax]) + ((double)r + 0.5) * a.inv_H * a.V[ax] - a.mo[ax]) *
               a.inv_h[ax];
    if (fabs(q - rint(q)) <= a.near_int[ax]) {
        const double p = __dadd_rn(__dadd_rn(a.o[ax], __dmul_rn(frac_of(c, a.W), a.U[ax])),
                                   __dmul_rn(frac_of(r, a.H), a.V[ax]));
        q = __ddiv_rn(__dsub_rn(p, a.mo[ax]), a.h[ax]);
    }
    double e = floor(q);
    if (e == (double)a.n[ax] && q == e) e -= 1.0;  // the top face belongs to the last element
    if (!(e >= 0.0 && e < (double)a.n[ax])) return -1;
    xi = 2.0 * (q - e) - 1.0;
    return (int)e;
}

// Axis path: element index of column (side 0) or row (side 1) c along its
// lattice axis, -1 outside.  q = A + (c + 0.5) B in FP32 differs from the
// correctly rounded FP64 q by less than thr_f / 4, so its floor is the exact
// one unless q lies within thr_f of an integer; there the FP64 rule decides.
__device__ __forceinline__ int own_axis(const SliceArgs& a, int side, int c) {
    const int ax = side == 0 ? a.ax_a : a.ax_b;
    const float qf = fmaf((float)c + 0.5f, a.Bf[side], a.Af[side]);
    if (fabsf(qf - rintf(qf)) <= a.thr_f[side]) {
        double xi;
        return locate_axis(a, ax, side == 0 ? c : 0, side == 0 ? 0 : c, xi);
    }
    const float ef = floorf(qf);
    return (ef >= 0.0f && ef < (float)a.n[ax]) ? (int)ef : -1;
}

// Reference coordinate of column (row) c in element e along its axis (FP64
// q, accurate to ~1e-15; it feeds the FP32 basis).
__device__ __forceinline__ float ref_coord(const SliceArgs& a, int side, int c, int e) {
    return (float)(2.0 * (fma((double)c + 0.5, a.Bd[side], a.Ad[side]) - (double)e) - 1.0);
}

// Lagrange basis through the GLL nodes at x: prefix and suffix products of
// (x - x_m) times the precomputed inverse denominators.
template <int LX>
__device__ __forceinline__ void basis(const SliceArgs& a, float x, float* L, int stride = 1) {
    float d[LX], pre[LX];
    float acc = 1.0f;
#pragma unroll
    for (int m = 0; m < LX; ++m) {
        d[m] = x - a.xn[m];
        pre[m] = acc;
        acc *= d[m];
    }
    float suf = 1.0f;
#pragma unroll
    for (int i = LX - 1; i >= 0; --i) {
        L[i * stride] = a.lw[i] * pre[i] * suf;
        suf *= d[i];
    }
}

// Bounds build: the slice kernels have no status word of their own, so a skipped access is
// recorded here (read and reset by semr_bounds_status).
__device__ unsigned g_slice_bounds;

__device__ __forceinline__ bool pixel_ok(const SliceArgs& a, int c, int r) {
    return bchk(c >= 0 && c < a.W && r >= 0 && r < a.H, &g_slice_bounds);
}
__device__ __forceinline__ bool element_ok(const SliceArgs& a, int64_t e) {
    return bchk(e >= 0 && e < (int64_t)a.n[0] * a.n[1] * a.n[2], &g_slice_bounds);
}

// Step 4 and the stores.  s: the coloured scalar (finite inside the mesh).
__device__ __forceinline__ void put_pixel(const SliceArgs& a, int c, int r, float s) {
    if (!pixel_ok(a, c, r)) return;
    float t = (s - a.vmin) * a.inv_range;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    int k = 0;
    while (k < a.n_ctrl - 2 && t >= a.ct[k + 1]) ++k;
    const float fk = (t - a.ct[k]) * a.cinvw[k];
    const float cr = fmaf(fk, a.dr[k], a.cr[k]);
    const float cg = fmaf(fk, a.dg[k], a.cg[k]);
    const float cb = fmaf(fk, a.db[k], a.cb[k]);
    auto byte = [](float v) -> unsigned {
        const int b = (int)floorf(fmaf(255.0f, v, 0.5f));
        return (unsigned)min(max(b, 0), 255);
    };
    const size_t px = (size_t)r * a.W + c;
    reinterpret_cast<uint32_t*>(a.rgba)[px] = byte(cr) | (byte(cg) << 8) | (byte(cb) << 16) | (255u << 24);
    if (a.values) a.values[px] = s;
}

__device__ __forceinline__ void put_background(const SliceArgs& a, int c, int r) {
    if (!pixel_ok(a, c, r)) return;
    const size_t px = (size_t)r * a.W + c;
    reinterpret_cast<uint32_t*>(a.rgba)[px] = a.bg;
    if (a.values) a.values[px] = __int_as_float(0x7fc00000);  // NaN
}

// ------------------------------------------------------------ axis-aligned

template <int LX>
__global__ void __launch_bounds__(kAxisThreads) slice_axis_kernel(const SliceArgs a) {
    constexpr int N2 = LX * LX, N3 = LX * LX * LX, LP = LX + 1;
    __shared__ float su[kMaxComp * N3];   // element values, one block per component
    __shared__ float sv[kMaxComp * N2];   // contracted along the normal: [comp][row-axis idx][col-axis idx]
    __shared__ float colL[kChunk * LP];   // basis values of a chunk of columns (padded rows)
    __shared__ float rowL[kChunk * LP];
    __shared__ float sw[kMaxComp * kChunk * LP];  // rows of a chunk contracted: [comp][row][col-axis idx]
    __shared__ int s_rng[4];              // first and last column, first and last row owned
    __shared__ int s_win[4];              // candidate windows (first, last) of columns and rows
    __shared__ float s_xi[2 * kWinCache];  // reference coordinates of the window's owned columns, rows

    const int tid = threadIdx.x;
    const int ea = a.ea0 + (int)(blockIdx.x % (unsigned)a.na);
    const int eb = a.eb0 + (int)(blockIdx.x / (unsigned)a.na);
    if (tid < 2) {  // candidate window per side: the element's extent in pixels, widened by 2
        const int side = tid;
        const int ax = side == 0 ? a.ax_a : a.ax_b;
        const int me = side == 0 ? ea : eb;
        const int npx = side == 0 ? a.W : a.H;
        const double o = a.o[ax], k = a.px_per[side];
        const double x0 = a.mo[ax] + me * a.h[ax], x1 = x0 + a.h[ax];
        double c0 = (x0 - o) * k - 0.5, c1 = (x1 - o) * k - 0.5;
        if (c0 > c1) {
            const double tmp = c0;
            c0 = c1;
            c1 = tmp;
        }
        c0 = fmax(fmin(floor(c0) - 2.0, (double)npx), -1.0);
        c1 = fmax(fmin(ceil(c1) + 2.0, (double)npx), -1.0);
        s_win[2 * side] = max((int)c0, 0);
        s_win[2 * side + 1] = min((int)c1, npx - 1);
        s_rng[2 * side] = INT_MAX;
        s_rng[2 * side + 1] = -1;
    }
    __syncthreads();
    // ---- the columns (rows) this element owns: an interval, since the
    // ownership rule is monotone in the column (row) index; the reference
    // coordinates of the window are kept for the basis when it is short
    for (int side = 0; side < 2; ++side) {
        const int me = side == 0 ? ea : eb;
        const int lo = s_win[2 * side], hi = s_win[2 * side + 1];
        for (int c = lo + tid; c <= hi; c += blockDim.x) {
            if (own_axis(a, side, c) == me) {
                atomicMin(&s_rng[2 * side], c);
                atomicMax(&s_rng[2 * side + 1], c);
                if (c - lo < kWinCache) s_xi[side * kWinCache + c - lo] = ref_coord(a, side, c, me);
            }
        }
    }
    __syncthreads();
    const int cfirst = s_rng[0], clast = s_rng[1], rfirst = s_rng[2], rlast = s_rng[3];
    if (clast < 0 || rlast < 0) return;  // uniform: the element owns no pixel

    // ---- load the element (all components) and contract along the normal
    auto coord = [&](int ax) { return ax == a.ax_a ? ea : (ax == a.ax_b ? eb : a.layer); };
    const int64_t e = coord(0) + (int64_t)a.n[0] * (coord(1) + (int64_t)a.n[1] * coord(2));
    if (!element_ok(a, e)) return;  // uniform over the CTA
    for (int comp = 0; comp < a.nc; ++comp) {
        const double* src = a.f[comp] + e * N3;
#pragma unroll 4
        for (int m = tid; m < N3; m += kAxisThreads) su[comp * N3 + m] = d2f_rz(__ldg(src + m));
    }
    __syncthreads();
    auto stride = [](int ax) { return ax == 0 ? 1 : (ax == 1 ? LX : N2); };  // of the i, j, k indices
    const int Sa = stride(a.ax_a), Sb = stride(a.ax_b), Sn = stride(a.ax_n);
    for (int i = tid; i < a.nc * N2; i += blockDim.x) {
        const int comp = i / N2, ib = (i % N2) / LX, ia = i % LX;
        const float* src = su + comp * N3 + ia * Sa + ib * Sb;
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < LX; ++t) acc = fmaf(a.Ln[t], src[t * Sn], acc);
        sv[i] = acc;
    }
    __syncthreads();

    // ---- pixels, in chunks of kChunk rows x kChunk columns.  Per row chunk
    // the rows are contracted first, w[comp][row][ia] = sum_ib l_ib(eta) v[comp][ib][ia],
    // so that a pixel costs lx FMAs per component.
    for (int r0 = rfirst; r0 <= rlast; r0 += kChunk) {
        const int nr = min(kChunk, rlast - r0 + 1);
        if (tid < nr) {
            const int r = r0 + tid, wi = r - s_win[2];
            float x;
            x = (wi < kWinCache) ? s_xi[kWinCache + wi] : ref_coord(a, 1, r, eb);
            basis<LX>(a, x, rowL + tid * LP);
        }
        __syncthreads();
        for (int i = tid; i < a.nc * nr * LX; i += blockDim.x) {
            const int comp = i / (nr * LX), rr = (i / LX) % nr, ia = i % LX;
            const float* v = sv + comp * N2 + ia;
            float acc = 0.0f;
#pragma unroll
            for (int ib = 0; ib < LX; ++ib) acc = fmaf(rowL[rr * LP + ib], v[ib * LX], acc);
            sw[(comp * kChunk + rr) * LP + ia] = acc;
        }
        __syncthreads();
        for (int c0 = cfirst; c0 <= clast; c0 += kChunk) {
            const int ncl = min(kChunk, clast - c0 + 1);
            if (tid < ncl) {
                const int c = c0 + tid, wi = c - s_win[0];
                float x;
                x = (wi < kWinCache) ? s_xi[wi] : ref_coord(a, 0, c, ea);
                basis<LX>(a, x, colL + tid * LP);
            }
            __syncthreads();
            // each thread keeps one column's basis in registers and walks rows
            const int per = kAxisThreads / ncl;  // rows per pass
            const int cc = tid % ncl, rsub = tid / ncl;
            if (rsub < per) {
                float cl[LX];
#pragma unroll
                for (int ia = 0; ia < LX; ++ia) cl[ia] = colL[cc * LP + ia];
                for (int rr = rsub; rr < nr; rr += per) {
                    float mag = 0.0f, s0 = 0.0f;
                    for (int comp = 0; comp < a.nc; ++comp) {
                        const float* w = sw + (comp * kChunk + rr) * LP;
                        float s = 0.0f;
#pragma unroll
                        for (int ia = 0; ia < LX; ++ia) s = fmaf(cl[ia], w[ia], s);
                        s0 = s;
                        mag = fmaf(s, s, mag);
                    }
                    put_pixel(a, c0 + cc, r0 + rr, a.nc == 1 ? s0 : sqrtf(mag));
                }
            }
            __syncthreads();
        }
    }
}

// Background for pixels that no element owns (only launched when the image
// reaches outside the lattice, or the plane misses it).
__global__ void __launch_bounds__(256) slice_fill_kernel(const SliceArgs a) {
    const int c = blockIdx.x * 16 + (threadIdx.x & 15), r = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (c >= a.W || r >= a.H) return;
    bool inside = a.layer >= 0;
    if (inside) {
        double xi;
        inside = locate_axis(a, a.ax_a, c, 0, xi) >= 0 && locate_axis(a, a.ax_b, 0, r, xi) >= 0;
    }
    if (!inside) put_background(a, c, r);
}

// ------------------------------------------------------------ any plane

template <int LX>
__global__ void __launch_bounds__(256) slice_generic_kernel(const SliceArgs a) {
    constexpr int N2 = LX * LX, N3 = LX * LX * LX;
    const int c = blockIdx.x * 16 + (threadIdx.x & 15), r = blockIdx.y * 16 + (threadIdx.x >> 4);
    if (c >= a.W || r >= a.H) return;
    double xi[3] = {0.0, 0.0, 0.0};
    int ei[3];
    bool inside = true;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        ei[ax] = locate_axis(a, ax, c, r, xi[ax]);
        inside &= ei[ax] >= 0;
    }
    if (!inside) {
        put_background(a, c, r);
        return;
    }
    const int64_t e = ei[0] + (int64_t)a.n[0] * (ei[1] + (int64_t)a.n[1] * ei[2]);
    if (!element_ok(a, e)) return;
    float Lx[LX], Ly[LX], Lz[LX];
    basis<LX>(a, (float)xi[0], Lx);
    basis<LX>(a, (float)xi[1], Ly);
    basis<LX>(a, (float)xi[2], Lz);
    float mag = 0.0f, s0 = 0.0f;
    for (int comp = 0; comp < a.nc; ++comp) {
        const double* u = a.f[comp] + e * N3;
        float s = 0.0f;
        for (int k = 0; k < LX; ++k) {
            float sj = 0.0f;
#pragma unroll
            for (int j = 0; j < LX; ++j) {
                float si = 0.0f;
#pragma unroll
                for (int i = 0; i < LX; ++i) si = fmaf(Lx[i], d2f_rz(__ldg(u + k * N2 + j * LX + i)), si);
                sj = fmaf(Ly[j], si, sj);
            }
            s = fmaf(Lz[k], sj, s);
        }
        s0 = s;
        mag = fmaf(s, s, mag);
    }
    put_pixel(a, c, r, a.nc == 1 ? s0 : sqrtf(mag));
}

// ------------------------------------------------------------ host side

bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

// Host FP64 version of the ownership rule (same operations, same order).
int locate_host(const SliceArgs& a, int ax, double fc, double fr, double* xi) {
    volatile double p = a.o[ax] + fc * a.U[ax];
    p = p + fr * a.V[ax];
    const double q = (p - a.mo[ax]) / a.h[ax];
    double e = std::floor(q);
    if (e == (double)a.n[ax] && q == e) e -= 1.0;
    if (!(e >= 0.0 && e < (double)a.n[ax])) return -1;
    if (xi) *xi = 2.0 * (q - e) - 1.0;
    return (int)e;
}

template <int LX>
int launch_slice(const SliceArgs& a, bool axis, bool fill, cudaStream_t st) {
    if (axis) {
        if (fill) {
            dim3 g((a.W + 15) / 16, (a.H + 15) / 16);
            slice_fill_kernel<<<g, 256, 0, st>>>(a);
        }
        if (a.layer >= 0 && a.na > 0 && a.nb > 0)
            slice_axis_kernel<LX><<<(unsigned)a.na * (unsigned)a.nb, kAxisThreads, 0, st>>>(a);
    } else {
        dim3 g((a.W + 15) / 16, (a.H + 15) / 16);
        slice_generic_kernel<LX><<<g, 256, 0, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? SEMR_OK : SEMR_ECUDA;
}

}  // namespace
}  // namespace semr

using namespace semr;

extern "C" int semr_slice_rgba(const semr_lattice* mesh, const double* const* fields, const semr_slice* sl,
                               uint8_t* rgba, float* values, void* cuda_stream) {
    if (!mesh || !fields || !sl || !rgba) return SEMR_EINVAL;
    if (mesh->lx < SEMR_LX_MIN || mesh->lx > SEMR_LX_MAX) return SEMR_EUNSUPPORTED;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) return SEMR_EINVAL;
    if ((int64_t)mesh->nx * mesh->ny * mesh->nz >= (1ll << 31)) return SEMR_EINVAL;
    if (!finite3(mesh->origin) || !finite3(mesh->h)) return SEMR_EINVAL;
    if (!(mesh->h[0] > 0.0 && mesh->h[1] > 0.0 && mesh->h[2] > 0.0)) return SEMR_EINVAL;
    if (sl->width < 1 || sl->height < 1 || sl->width > SEMR_SLICE_MAX_SIDE || sl->height > SEMR_SLICE_MAX_SIDE)
        return SEMR_EINVAL;
    if (sl->n_comp < 1 || sl->n_comp > SEMR_SLICE_MAX_COMP) return SEMR_EINVAL;
    if (sl->n_ctrl < 2 || sl->n_ctrl > SEMR_SLICE_MAX_CTRL) return SEMR_EINVAL;
    if (!finite3(sl->origin) || !finite3(sl->axis_u) || !finite3(sl->axis_v)) return SEMR_EINVAL;
    if (!std::isfinite(sl->vmin) || !std::isfinite(sl->vmax) || !(sl->vmax > sl->vmin)) return SEMR_EINVAL;
    if (sl->ctrl[0][0] != 0.0 || sl->ctrl[sl->n_ctrl - 1][0] != 1.0) return SEMR_EINVAL;
    for (int k = 0; k < sl->n_ctrl; ++k) {
        if (k > 0 && !(sl->ctrl[k][0] > sl->ctrl[k - 1][0])) return SEMR_EINVAL;
        for (int c = 1; c < 4; ++c)
            if (!(sl->ctrl[k][c] >= 0.0 && sl->ctrl[k][c] <= 1.0)) return SEMR_EINVAL;
    }
    if ((reinterpret_cast<uintptr_t>(rgba) & 3u) || (reinterpret_cast<uintptr_t>(values) & 3u)) return SEMR_EINVAL;
    const uintptr_t amask = (mesh->lx % 2 == 0) ? 15u : 7u;
    for (int c = 0; c < sl->n_comp; ++c)
        if (!fields[c] || (reinterpret_cast<uintptr_t>(fields[c]) & amask)) return SEMR_EINVAL;

    SliceArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int c = 0; c < sl->n_comp; ++c) a.f[c] = fields[c];
    a.rgba = rgba;
    a.values = values;
    a.lx = mesh->lx;
    a.nc = sl->n_comp;
    a.n[0] = mesh->nx;
    a.n[1] = mesh->ny;
    a.n[2] = mesh->nz;
    for (int d = 0; d < 3; ++d) {
        a.mo[d] = mesh->origin[d];
        a.h[d] = mesh->h[d];
        a.o[d] = sl->origin[d];
        a.U[d] = sl->axis_u[d];
        a.V[d] = sl->axis_v[d];
    }
    a.W = sl->width;
    a.H = sl->height;
    a.vmin = (float)sl->vmin;
    a.inv_range = (float)(1.0 / (sl->vmax - sl->vmin));
    a.n_ctrl = sl->n_ctrl;
    for (int k = 0; k < sl->n_ctrl; ++k) {
        a.ct[k] = (float)sl->ctrl[k][0];
        a.cinvw[k] = k + 1 < sl->n_ctrl ? (float)(1.0 / (sl->ctrl[k + 1][0] - sl->ctrl[k][0])) : 0.0f;
        a.cr[k] = (float)sl->ctrl[k][1];
        a.cg[k] = (float)sl->ctrl[k][2];
        a.cb[k] = (float)sl->ctrl[k][3];
    }
    for (int k = 0; k + 1 < sl->n_ctrl; ++k) {
        a.dr[k] = a.cr[k + 1] - a.cr[k];
        a.dg[k] = a.cg[k + 1] - a.cg[k];
        a.db[k] = a.cb[k + 1] - a.cb[k];
    }
    a.bg = sl->background;
    a.inv_W = 1.0 / a.W;
    a.inv_H = 1.0 / a.H;
    for (int d = 0; d < 3; ++d) {
        a.inv_h[d] = 1.0 / a.h[d];
        // the fast q differs from the correctly rounded one by a few units of 2^-52 times
        // (|o| + |U| + |V| + |mo|) / h; far below this margin
        a.near_int[d] = 1e-11 * (1.0 + (std::fabs(a.o[d]) + std::fabs(a.U[d]) + std::fabs(a.V[d]) +
                                        std::fabs(a.mo[d])) / a.h[d]);
    }
    const int lx = mesh->lx;
    double xn[SEMR_LX_MAX], wq[SEMR_LX_MAX];
    if (gll_nodes_weights(lx, xn, wq) != 0) return SEMR_EINVAL;
    double lw[SEMR_LX_MAX];
    for (int i = 0; i < lx; ++i) {
        double d = 1.0;
        for (int m = 0; m < lx; ++m)
            if (m != i) d *= xn[i] - xn[m];
        lw[i] = 1.0 / d;
        a.xn[i] = (float)xn[i];
        a.lw[i] = (float)lw[i];
    }

    // axis-aligned slice: axis_u and axis_v each along one, different, lattice axis
    int ua = -1, va = -1, nu = 0, nv = 0;
    for (int d = 0; d < 3; ++d) {
        if (sl->axis_u[d] != 0.0) ua = d, ++nu;
        if (sl->axis_v[d] != 0.0) va = d, ++nv;
    }
    const bool axis = nu == 1 && nv == 1 && ua != va;
    bool fill = false;
    if (axis) {
        a.ax_a = ua;
        a.ax_b = va;
        a.ax_n = 3 - ua - va;
        a.px_per[0] = a.W / a.U[ua];
        a.px_per[1] = a.H / a.V[va];
        for (int side = 0; side < 2; ++side) {
            const int ax = side == 0 ? ua : va;
            const double w = side == 0 ? a.U[ua] : a.V[va];
            const double npx = side == 0 ? a.W : a.H;
            a.Ad[side] = (a.o[ax] - a.mo[ax]) / a.h[ax];
            a.Bd[side] = w / (npx * a.h[ax]);
            a.Af[side] = (float)a.Ad[side];
            a.Bf[side] = (float)a.Bd[side];
            // |q_f - q| <= 2^-23 (|A| + npx |B|) + 2^-24 |q| < 2^-22 (|A| + |w| / h); four times that margin
            a.thr_f[side] = (float)(std::ldexp(1.0, -20) * (1.0 + std::fabs(a.Ad[side]) + std::fabs(w) / a.h[ax]));
        }
        double zeta = 0.0;
        a.layer = locate_host(a, a.ax_n, 0.5, 0.5, &zeta);
        if (a.layer >= 0) {
            for (int t = 0; t < lx; ++t) {  // l_t(zeta), product definition in FP64
                double v = 1.0;
                for (int m = 0; m < lx; ++m)
                    if (m != t) v *= (zeta - xn[m]) / (xn[t] - xn[m]);
                a.Ln[t] = (float)v;
            }
            // elements of the layer that the image's first and last columns (rows) reach;
            // the rule is monotone, so every owned pixel lies between them
            auto range = [&](int ax, bool col, int npx, int* e0, int* cnt) {
                const int nax = a.n[ax];
                double q0 = (sl->origin[ax] - mesh->origin[ax]) / mesh->h[ax];
                double q1 = (sl->origin[ax] + (col ? sl->axis_u[ax] : sl->axis_v[ax]) - mesh->origin[ax]) / mesh->h[ax];
                if (q0 > q1) std::swap(q0, q1);
                const double lo = std::floor(q0) - 1.0, hi = std::floor(q1) + 1.0;  // clamp before converting
                const int l = (int)std::fmin(std::fmax(lo, 0.0), (double)nax);
                const int h = (int)std::fmax(std::fmin(hi, (double)(nax - 1)), -1.0);
                *e0 = l;
                *cnt = h >= l ? h - l + 1 : 0;
                (void)npx;
            };
            range(a.ax_a, true, a.W, &a.ea0, &a.na);
            range(a.ax_b, false, a.H, &a.eb0, &a.nb);
            // every pixel inside when the extreme columns and rows are (monotone rule)
            fill = locate_host(a, a.ax_a, 0.5 / a.W, 0.5, nullptr) < 0 ||
                   locate_host(a, a.ax_a, (a.W - 0.5) / a.W, 0.5, nullptr) < 0 ||
                   locate_host(a, a.ax_b, 0.5, 0.5 / a.H, nullptr) < 0 ||
                   locate_host(a, a.ax_b, 0.5, (a.H - 0.5) / a.H, nullptr) < 0;
        } else {
            fill = true;
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    switch (lx) {
        case 2: return launch_slice<2>(a, axis, fill, st);
        case 3: return launch_slice<3>(a, axis, fill, st);
        case 4: return launch_slice<4>(a, axis, fill, st);
        case 5: return launch_slice<5>(a, axis, fill, st);
        case 6: return launch_slice<6>(a, axis, fill, st);
        case 7: return launch_slice<7>(a, axis, fill, st);
        case 8: return launch_slice<8>(a, axis, fill, st);
        case 9: return launch_slice<9>(a, axis, fill, st);
        case 10: return launch_slice<10>(a, axis, fill, st);
        case 11: return launch_slice<11>(a, axis, fill, st);
        case 12: return launch_slice<12>(a, axis, fill, st);
        default: return SEMR_EUNSUPPORTED;
    }
}

extern "C" uint32_t semr_bounds_status(int reset) {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, semr::g_slice_bounds, sizeof(v)) != cudaSuccess) return 0xffffffffu;
    if (reset) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(semr::g_slice_bounds, &z, sizeof(z)) != cudaSuccess) return 0xffffffffu;
    }
    return v;
}
