// pip_raster.cu -- pixel coverage of a batch of convex polygons (the
// screen-space use of the inclusion test, Sec. 1: every pixel's membership is
// decided by a point inclusion test): for each pixel centre, the lowest-index
// polygon whose closed polygon holds it (front to back), and a coverage mask.
//
// Pixel (c, r) has the float32 centre (fmaf(c, dx, x0), fmaf(r, dy, y0)): one
// rounding each, so a point set identical to materialising those centres and
// calling the all-pairs test.
//
// 1. raster_bin_kernel: one thread per polygon marks the 64 x 48 tiles its
//    vertex bounding box can reach, in a tile x polygon bitmask.
// 2. raster_tile_kernel: one CTA per tile; thread t holds 12 pixels (a warp a
//    64 x 6 strip), walks the tile's polygons in index order (the bitmask
//    compacted into a shared list), skips a polygon for a warp whose strip
//    misses its bounding box, and evaluates the float32 test (Eq. 11
//    expanded, running min, error bound) otherwise; a warp stops once each of
//    its pixels has a candidate (decided inside, or uncertain).  The warp then
//    decides each of its uncertain pixels exactly (refine_pixel: the tile's
//    polygons upward from the candidate, float32 decision per polygon, fp64
//    Voronoi and exact orientation where it is uncertain) and writes the ids
//    and the mask words (32 aligned columns of a row per ballot).
#include <float.h>
#include <math.h>

#include "pip_kernels.cuh"
#include "pip_tma.cuh"

using namespace pip;

namespace {

constexpr int kRtW = 64, kRtH = 48;  // tile of pixels
constexpr int kRtThreads = 256;      // 8 warps; warp w: rows 6w .. 6w + 5
constexpr int kRtPT = 12;            // pixels per thread: 2 columns x 6 rows

struct RasterGrid {
    int W, H, tiles_x, tiles_y, words;  // words: polygon-bitmask words per tile
    float x0, y0, dx, dy;
};

__device__ __forceinline__ float centre_x(const RasterGrid &g, int c) { return fmaf((float)c, g.dx, g.x0); }
__device__ __forceinline__ float centre_y(const RasterGrid &g, int r) { return fmaf((float)r, g.dy, g.y0); }

// Tiles that may hold a pixel centre inside polygon j's bounding box (a
// conservative index range: the exact test happens per warp later).
__global__ void raster_bin_kernel(const PolyInfo *__restrict__ poly, int P, RasterGrid g,
                                  uint32_t *__restrict__ bits)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const PolyInfo pi = poly[j];
    if (pi.status != PIP_OK) return;
    const double cx0 = floor(((double)pi.bbox[0] - g.x0) / g.dx) - 1.0;
    const double cx1 = ceil(((double)pi.bbox[2] - g.x0) / g.dx) + 1.0;
    const double cy0 = floor(((double)pi.bbox[1] - g.y0) / g.dy) - 1.0;
    const double cy1 = ceil(((double)pi.bbox[3] - g.y0) / g.dy) + 1.0;
    if (!(cx1 >= 0.0 && cy1 >= 0.0 && cx0 <= g.W - 1.0 && cy0 <= g.H - 1.0)) return;
    const int tx0 = (int)fmax(cx0, 0.0) / kRtW, tx1 = (int)fmin(cx1, g.W - 1.0) / kRtW;
    const int ty0 = (int)fmax(cy0, 0.0) / kRtH, ty1 = (int)fmin(cy1, g.H - 1.0) / kRtH;
    const uint32_t bit = 1u << (j & 31);
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx)
            atomicOr(&bits[((size_t)ty * g.tiles_x + tx) * g.words + (j >> 5)], bit);
}

__device__ __forceinline__ float rs(const float4 &c, float x, float y) { return fmaf(-x, c.x, fmaf(-y, c.y, c.z)); }

// float32 decision of polygon j at a point: 1 inside, 0 uncertain, -1 outside
__device__ int decide_xy(const PolyInfo &pi, const float4 *__restrict__ coefp, int j, float px, float py)
{
    if (pi.status != PIP_OK) return -1;
    const float x = px - pi.ox, y = py - pi.oy;
    const float4 *cf = coefp + (size_t)j * kPadStride;
    float m = INFINITY;
    for (int k = 0; k < pi.n; ++k) m = fmin_nan(m, rs(cf[k], x, y));
    const float B = fmaf(pi.beta1, fabsf(x) + fabsf(y), pi.beta0);
    if (m >= B) return 1;
    return !(fabsf(m) >= B) ? 0 : -1;
}

// Exact first hit of one pixel, by the whole warp (every lane passes the same
// arguments): the tile's polygons from `start` upward, 32 bitmask words per
// step (one per lane), then each non-empty word's polygons with lane l taking
// its l-th set bit: float32 decision per polygon, and for an uncertain one the
// exact re-decision (fp64 Voronoi, then exact orientation).  -1 if none.
__device__ __noinline__ int refine_pixel(const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefp,
                                         const double2 *__restrict__ g0, const double2 *__restrict__ gk,
                                         const void *__restrict__ verts, int vdtype, int words,
                                         const uint32_t *__restrict__ tb, int start, float px, float py)
{
    const int lane = threadIdx.x & 31;
    for (int wb = start >> 5; wb < words; wb += 32) {
        const int wl = wb + lane;
        uint32_t mine = wl < words ? tb[wl] : 0u;
        if (wl == (start >> 5)) mine &= ~0u << (start & 31);
        uint32_t nz = __ballot_sync(0xffffffffu, mine != 0u);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            const uint32_t word = __shfl_sync(0xffffffffu, mine, src);
            uint32_t rest = word;
            for (int t = 0; t < lane && rest; ++t) rest &= rest - 1;
            const int j = rest ? 32 * (wb + src) + __ffs(rest) - 1 : -1;
            const int b = j >= 0 ? decide_xy(poly[j], coefp, j, px, py) : -1;
            const uint32_t in_m = __ballot_sync(0xffffffffu, b > 0);
            uint32_t cand = in_m | __ballot_sync(0xffffffffu, b == 0);
            while (cand) {  // lanes are in polygon order
                const int l = __ffs(cand) - 1;
                cand &= cand - 1;
                const int jl = __shfl_sync(0xffffffffu, j, l);
                if ((in_m >> l) & 1u) return jl;
                const PolyInfo pl = poly[jl];
                if (warp_inside_exact_xy(pl, jl, g0, gk, verts, vdtype, (double)px, (double)py)) return jl;
            }
        }
    }
    return -1;
}

__global__ void __launch_bounds__(kRtThreads, 2) raster_tile_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefp, RasterGrid g,
    const uint32_t *__restrict__ bits, const double2 *__restrict__ g0, const double2 *__restrict__ gk,
    const void *__restrict__ verts, int vdtype, int32_t *__restrict__ ids, uint32_t *__restrict__ mask,
    unsigned int *__restrict__ refined)
{
    const int tx = blockIdx.x % g.tiles_x, ty = blockIdx.x / g.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = tx * kRtW, r0 = ty * kRtH + 6 * warp;
    float px[kRtPT], py[kRtPT];
    uint32_t key[kRtPT];
    bool live[kRtPT];
#pragma unroll
    for (int i = 0; i < kRtPT; ++i) {
        const int c = c0 + lane + 32 * (i & 1), r = r0 + (i >> 1);
        live[i] = c < g.W && r < g.H;
        px[i] = centre_x(g, c);
        py[i] = centre_y(g, r);
        key[i] = live[i] ? 0xffffffffu : 0u;  // a pixel outside the frame counts as settled
    }
    // the warp's strip of centres (monotone in c and r: dx, dy > 0)
    const float sx0 = centre_x(g, c0), sx1 = centre_x(g, min(c0 + kRtW, g.W) - 1);
    const float sy0 = centre_y(g, min(r0, g.H - 1)), sy1 = centre_y(g, min(r0 + 5, g.H - 1));
    const uint32_t *tb = bits + (size_t)blockIdx.x * g.words;
    bool done = r0 >= g.H;
    // The tile's polygons in index order: kRtThreads bitmask words at a time,
    // one per thread, compacted by a block prefix sum into a shared list.
    __shared__ uint16_t s_list[kRtThreads * 32];
    __shared__ int s_warp_tot[kRtThreads / 32];
    for (int wbase = 0; wbase < g.words; wbase += kRtThreads) {
        const int wd = wbase + threadIdx.x;
        uint32_t word = wd < g.words ? tb[wd] : 0u;
        const int cnt = __popc(word);
        int incl = cnt;  // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        __syncthreads();  // every warp is done with the previous list
        if (lane == 31) s_warp_tot[warp] = incl;
        __syncthreads();
        int before = 0, total = 0;
        for (int w2 = 0; w2 < kRtThreads / 32; ++w2) {
            const int t = s_warp_tot[w2];
            before += w2 < warp ? t : 0;
            total += t;
        }
        int at = before + incl - cnt;
        while (word) {
            s_list[at++] = (uint16_t)(32 * threadIdx.x + __ffs(word) - 1);
            word &= word - 1;
        }
        __syncthreads();
        for (int e = 0; e < total && !done; ++e) {
            const int j = 32 * wbase + s_list[e];
            const PolyInfo pi = poly[j];
            if (pi.bbox[0] > sx1 || pi.bbox[2] < sx0 || pi.bbox[1] > sy1 || pi.bbox[3] < sy0) continue;
            bool open = false;
#pragma unroll
            for (int i = 0; i < kRtPT; ++i)
                open |= key[i] == 0xffffffffu && px[i] >= pi.bbox[0] && px[i] <= pi.bbox[2] &&
                        py[i] >= pi.bbox[1] && py[i] <= pi.bbox[3];
            if (!__any_sync(0xffffffffu, open)) continue;
            const float4 *cf = coefp + (size_t)j * kPadStride;
            const int n = pi.n;  // at least 3
            float x[kRtPT], y[kRtPT], m[kRtPT];
            {
                const float4 a = cf[0], b = cf[1], c = cf[2];
#pragma unroll
                for (int i = 0; i < kRtPT; ++i) {
                    x[i] = px[i] - pi.ox;
                    y[i] = py[i] - pi.oy;
                    m[i] = fmin3_nan(rs(a, x[i], y[i]), rs(b, x[i], y[i]), rs(c, x[i], y[i]));
                }
            }
            int k = 3;
            for (; k + 4 <= n; k += 4) {
                const float4 a = cf[k], b = cf[k + 1], c = cf[k + 2], d = cf[k + 3];
#pragma unroll
                for (int i = 0; i < kRtPT; ++i)
                    m[i] = fmin3_nan(fmin3_nan(m[i], rs(a, x[i], y[i]), rs(b, x[i], y[i])), rs(c, x[i], y[i]),
                                     rs(d, x[i], y[i]));
            }
            for (; k < n; ++k) {
                const float4 a = cf[k];
#pragma unroll
                for (int i = 0; i < kRtPT; ++i) m[i] = fmin_nan(m[i], rs(a, x[i], y[i]));
            }
            const uint32_t jj = (uint32_t)j << 1;
            bool settled = true;
#pragma unroll
            for (int i = 0; i < kRtPT; ++i) {
                const float B = fmaf(pi.beta1, fabsf(x[i]) + fabsf(y[i]), pi.beta0);
                const bool in = m[i] >= B;
                const bool unc = !(fabsf(m[i]) >= B);
                if (key[i] == 0xffffffffu && (in || unc)) key[i] = jj | (in ? 0u : 1u);
                settled &= key[i] != 0xffffffffu;
            }
            done = __all_sync(0xffffffffu, settled);  // later polygons cannot lower any key
        }
    }
    // Outputs of the decided pixels.  Pixel group i of the warp is 32
    // consecutive columns of one row starting at a multiple of 32: one mask
    // word.  An uncertain pixel is written as outside here and corrected below.
    const int wpr = (g.W + 31) / 32;
    __shared__ uint32_t s_keys[kRtThreads / 32][kRtPT][32];
#pragma unroll
    for (int i = 0; i < kRtPT; ++i) {
        const int cg = c0 + 32 * (i & 1), r = r0 + (i >> 1);
        const bool in = live[i] && key[i] != 0xffffffffu && !(key[i] & 1u);
        if (live[i] && ids) ids[(size_t)r * g.W + cg + lane] = in ? (int32_t)(key[i] >> 1) : -1;
        const uint32_t word = __ballot_sync(0xffffffffu, in);
        if (mask && lane == 0 && r < g.H && cg < g.W) mask[(size_t)r * wpr + cg / 32] = word;
        s_keys[warp][i][lane] = live[i] ? key[i] : 0xffffffffu;
    }
    __syncwarp();
    // Uncertain pixels (rare): the warp decides each exactly, in turn.
#pragma unroll 1
    for (int i = 0; i < kRtPT; ++i) {
        const uint32_t k = s_keys[warp][i][lane];
        uint32_t u = __ballot_sync(0xffffffffu, k != 0xffffffffu && (k & 1u));
        if (u && lane == 0) atomicAdd(refined, (unsigned int)__popc(u));
        while (u) {
            const int l = __ffs(u) - 1;
            u &= u - 1;
            const int start = (int)(__shfl_sync(0xffffffffu, k, l) >> 1);
            const int c = c0 + 32 * (i & 1) + l, r = r0 + (i >> 1);
            const int hit = refine_pixel(poly, coefp, g0, gk, verts, vdtype, g.words, tb, start, centre_x(g, c),
                                         centre_y(g, r));
            if (lane == 0) {
                if (ids) ids[(size_t)r * g.W + c] = hit;
                if (mask && hit >= 0) atomicOr(&mask[(size_t)r * wpr + c / 32], 1u << (c & 31));
            }
        }
    }
}

bool grid_ok(int32_t W, int32_t H, float x0, float y0, float dx, float dy)
{
    return W >= 1 && H >= 1 && isfinite(x0) && isfinite(y0) && isfinite(dx) && isfinite(dy) && dx > 0.f &&
           dy > 0.f && isfinite(fmaf((float)(W - 1), dx, x0)) && isfinite(fmaf((float)(H - 1), dy, y0)) &&
           W <= (1 << 24) && H <= (1 << 24);
}

RasterGrid make_grid(int P, int32_t W, int32_t H, float x0, float y0, float dx, float dy)
{
    RasterGrid g;
    g.W = W;
    g.H = H;
    g.tiles_x = (W + kRtW - 1) / kRtW;
    g.tiles_y = (H + kRtH - 1) / kRtH;
    g.words = (P + 31) / 32;
    g.x0 = x0;
    g.y0 = y0;
    g.dx = dx;
    g.dy = dy;
    return g;
}

}  // namespace

extern "C" size_t pip_raster_workspace_bytes(int32_t num_polygons, int32_t width, int32_t height)
{
    if (num_polygons < 1 || width < 1 || height < 1) return 0;
    const size_t tiles = (size_t)((width + kRtW - 1) / kRtW) * (size_t)((height + kRtH - 1) / kRtH);
    return tiles * (size_t)((num_polygons + 31) / 32) * sizeof(uint32_t);
}

extern "C" pip_status pip_rasterize(const pip_tables *t, int32_t width, int32_t height, float x0, float y0,
                                    float dx, float dy, int32_t *d_first_hit, uint32_t *d_mask,
                                    void *d_workspace, size_t workspace_bytes, void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (!grid_ok(width, height, x0, y0, dx, dy)) return PIP_E_INVALID_ARG;
    if (d_first_hit == nullptr && d_mask == nullptr) return PIP_E_INVALID_ARG;
    if ((d_first_hit && !aligned(d_first_hit, 4)) || (d_mask && !aligned(d_mask, 4))) return PIP_E_INVALID_ARG;
    const size_t need = pip_raster_workspace_bytes(t->P, width, height);
    if (d_workspace == nullptr || !aligned(d_workspace, 16) || workspace_bytes < need) return PIP_E_INVALID_ARG;
    if ((int64_t)width * height > t->capacity) return PIP_E_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    const RasterGrid g = make_grid(t->P, width, height, x0, y0, dx, dy);
    uint32_t *bits = (uint32_t *)d_workspace;
    PIP_CUDA_TRY(cudaMemsetAsync(bits, 0, need, s));
    PIP_CUDA_TRY(cudaMemsetAsync(t->d_qcount, 0, sizeof(unsigned int), s));
    raster_bin_kernel<<<(t->P + 255) / 256, 256, 0, s>>>(t->d_poly, t->P, g, bits);
    PIP_CUDA_TRY(cudaGetLastError());
    timing_mark(t, 0, s);
    raster_tile_kernel<<<g.tiles_x * g.tiles_y, kRtThreads, 0, s>>>(t->d_poly, t->d_coefp, g, bits, t->d_g0,
                                                                   t->d_gk, t->d_verts, t->vdtype, d_first_hit,
                                                                   d_mask, t->d_qcount);
    PIP_CUDA_TRY(cudaGetLastError());
    timing_mark(t, 1, s);
    timing_mark(t, 2, s);
    return PIP_OK;
}
