// pip_compare.cu -- the paper's two reference tests and the plain fp64 form of
// Alg. 5, as GPU kernels, so that all three compare on the same chip.
//
//   sign of offset (Alg. 2, float32): dV = V - V', LHS = q_y dV_x - q_x dV_y,
//       RHS = V'_y dV_x - V'_x dV_y, D = LHS < RHS; inside when every D is equal
//       (sum D mod n = 0).
//   ray crossing   (Alg. 1, float32, +x ray): crossing when the edge straddles
//       q_y ((V_y > q_y) xor (V'_y > q_y)) and q is on the correct side
//       (LHS > RHS for an upward edge, LHS < RHS otherwise); an odd count is
//       inside (the text of Sec. 2.1; the listing's "= 0" is read as a typo).
//   plain fp64 Voronoi (Alg. 5): M_0 <= M_k for every k, M the squared
//       distances to the fp64 generators.  "Unbatched": one launch per polygon.
//
// None of these carries an error bound: each decides in its own precision, as
// the listings do.  Same chunk layout and mask packing as the main test.
#include <stdlib.h>

#include "pip_kernels.cuh"

using namespace pip;

namespace {

enum CmpOp { kSignOfOffset = 0, kRayCrossing = 1, kVoronoiFp64 = 2 };

struct CmpEdge {
    float4 a;   // sign of offset / ray: (dVx, dVy, RHS, going_up)
    float4 b;   // ray: (V'_y, V_y, 0, 0)
};

template <int OP>
__device__ __forceinline__ bool cmp_eval(float qx, float qy, const CmpEdge *e, const double2 *g, double2 g0,
                                         int n)
{
    if (OP == kSignOfOffset) {
        int sumD = 0;
        for (int k = 0; k < n; ++k) {
            const float4 c = e[k].a;
            const float lhs = qy * c.x - qx * c.y;
            sumD += lhs < c.z ? 1 : 0;
        }
        return sumD == 0 || sumD == n;  // sum mod n == 0
    } else if (OP == kRayCrossing) {
        int cross = 0;
        for (int k = 0; k < n; ++k) {
            const float4 c = e[k].a;
            const float4 d = e[k].b;
            const bool in_range = (d.y > qy) != (d.x > qy);
            const float lhs = qy * c.x - qx * c.y;
            const bool on_left = c.w != 0.f ? (lhs > c.z) : (lhs < c.z);
            cross += (in_range && on_left) ? 1 : 0;
        }
        return cross & 1;
    } else {
        const double x = (double)qx, y = (double)qy;
        const double d0x = x - g0.x, d0y = y - g0.y;
        const double M0 = d0x * d0x + d0y * d0y;
        bool in = true;
        for (int k = 0; k < n; ++k) {
            const double dx = x - g[k].x, dy = y - g[k].y;
            in &= M0 <= dx * dx + dy * dy;
        }
        return in;
    }
}

template <int OP, int F, bool V16>
__global__ void __launch_bounds__(kThreads) cmp_kernel(const PolyInfo *__restrict__ poly, int j,
                                                       const float *__restrict__ verts,
                                                       const double2 *__restrict__ g0tab,
                                                       const double2 *__restrict__ gktab,
                                                       const float *__restrict__ pts, int64_t M,
                                                       int64_t lo, int64_t hi, int64_t hi_w,
                                                       uint32_t *__restrict__ mask)
{
    __shared__ CmpEdge se[kMaxEdges];
    __shared__ double2 sg[kMaxEdges];
    const PolyInfo pi = poly[j];
    const bool ok = pi.status == PIP_OK;
    const int n = ok ? pi.n : 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int km = k == 0 ? n - 1 : k - 1;
        const float vx = verts[2 * (pi.voff + k)], vy = verts[2 * (pi.voff + k) + 1];
        const float ux = verts[2 * (pi.voff + km)], uy = verts[2 * (pi.voff + km) + 1];
        const float dvx = vx - ux, dvy = vy - uy;
        CmpEdge e;
        e.a = make_float4(dvx, dvy, uy * dvx - ux * dvy, vy > uy ? 1.f : 0.f);
        e.b = make_float4(uy, vy, 0.f, 0.f);
        se[k] = e;
        if (OP == kVoronoiFp64) sg[k] = gktab[pi.voff + k];
    }
    const double2 g0 = OP == kVoronoiFp64 && ok ? g0tab[j] : make_double2(0.0, 0.0);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t c_first = lo / Chunk<F>::kPoints;
    const int64_t c_end = hi > lo ? (hi - 1) / Chunk<F>::kPoints + 1 : c_first;
    for (int64_t c = c_first + warp; c < c_end; c += nwarps) {
        const int64_t p0 = c * Chunk<F>::kPoints;
        uint32_t myword = 0;
#pragma unroll
        for (int jj = 0; jj < F; ++jj) {
            const int64_t q2 = p0 + 2 * (jj * 32 + lane);
            float x0, y0, x1, y1;
            load_pair<false, V16>(pts, q2, M, x0, y0, x1, y1);
            const bool in0 = ok && q2 >= lo && q2 < hi && cmp_eval<OP>(x0, y0, se, sg, g0, n);
            const bool in1 = ok && q2 + 1 >= lo && q2 + 1 < hi && cmp_eval<OP>(x1, y1, se, sg, g0, n);
            uint32_t wl, wh;
            interleave_words(__ballot_sync(0xffffffffu, in0), __ballot_sync(0xffffffffu, in1), wl, wh);
            if (lane == 2 * jj) myword = wl;
            if (lane == 2 * jj + 1) myword = wh;
        }
        if (lane < 2 * F) {
            const int64_t w = (p0 >> 5) + lane;
            const int64_t first = w << 5;
            uint32_t own;
            if (first >= lo && first + 32 <= hi_w) {
                own = 0xffffffffu;
            } else {
                own = 0;
                for (int b = 0; b < 32; ++b)
                    if (first + b >= lo && first + b < hi_w) own |= 1u << b;
            }
            if (own == 0xffffffffu) {
                mask[w] = myword;
            } else if (own) {
                atomicAnd(&mask[w], ~own);
                atomicOr(&mask[w], myword & own);
            }
        }
    }
}

constexpr int kF = 4;

template <int OP>
pip_status run_cmp(const pip_tables *t, const float *d_points, int64_t M, const int64_t *d_point_offsets,
                   uint32_t *d_mask, void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (t->vdtype != PIP_F32) return PIP_E_INVALID_ARG;  // the listings take float vertices
    if (M < 0) return PIP_E_INVALID_ARG;
    if (M == 0) return PIP_OK;
    if (d_points == nullptr || d_mask == nullptr || !aligned(d_points, 8) || !aligned(d_mask, 4))
        return PIP_E_INVALID_ARG;
    if (d_point_offsets == nullptr && t->P != 1) return PIP_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool v16 = aligned(d_points, 16);
    auto k = v16 ? cmp_kernel<OP, kF, true> : cmp_kernel<OP, kF, false>;
    const int full = blocks_for(k, t->num_sms, kThreads);
    const int64_t hi_last = (M + 31) & ~(int64_t)31;
    auto launch = [&](int j, int64_t lo, int64_t hi, int64_t hi_w) -> cudaError_t {
        const int64_t chunks = hi > lo ? (hi - 1) / Chunk<kF>::kPoints - lo / Chunk<kF>::kPoints + 1 : 0;
        if (chunks == 0) return cudaSuccess;
        const int blocks = (int)max((int64_t)1, min((int64_t)full, (chunks + kWarps - 1) / kWarps));
        k<<<blocks, kThreads, 0, s>>>(t->d_poly, j, (const float *)t->d_verts, t->d_g0, t->d_gk,
                                      d_points, M, lo, hi, hi_w, d_mask);
        return cudaGetLastError();
    };
    if (d_point_offsets == nullptr) {
        // one polygon: sign of offset and ray crossing through the pipelined
        // single-polygon kernel (constant-bank edges, bulk-copy ring, ballot
        // packing: the Voronoi kernel's frame) when the points allow bulk
        // copies; the fp64 form and unaligned points take the register kernel
        if (OP != kVoronoiFp64 && v16 && t->have_host_poly) {
            PIP_CUDA_TRY(launch_cmp_stream(t, d_points, M, d_mask, OP == kSignOfOffset ? 1 : 2, s));
            return PIP_OK;
        }
        PIP_CUDA_TRY(launch(0, 0, M, hi_last));
        return PIP_OK;
    }
    // own-polygon batch: the pipelined batch kernel's schedule, offsets read on
    // the device (one sequence of launches, no host synchronisation)
    if (!v16) return PIP_E_INVALID_ARG;
    if (!aligned(d_point_offsets, 8)) return PIP_E_INVALID_ARG;
    if (M > t->capacity) return PIP_E_CAPACITY;
    PIP_CUDA_TRY(launch_ragged_cmp(t, d_points, M, d_point_offsets, d_mask,
                                   OP == kSignOfOffset ? 1 : OP == kRayCrossing ? 2 : 3, s));
    return PIP_OK;
}

}  // namespace

extern "C" {

pip_status pip_test_sign_of_offset(const pip_tables *t, const float *d_points, int64_t num_points,
                                   const int64_t *d_point_offsets, uint32_t *d_mask, void *stream)
{
    return run_cmp<kSignOfOffset>(t, d_points, num_points, d_point_offsets, d_mask, stream);
}

pip_status pip_test_ray_crossing(const pip_tables *t, const float *d_points, int64_t num_points,
                                 const int64_t *d_point_offsets, uint32_t *d_mask, void *stream)
{
    return run_cmp<kRayCrossing>(t, d_points, num_points, d_point_offsets, d_mask, stream);
}

pip_status pip_test_voronoi_fp64(const pip_tables *t, const float *d_points, int64_t num_points,
                                 const int64_t *d_point_offsets, uint32_t *d_mask, void *stream)
{
    return run_cmp<kVoronoiFp64>(t, d_points, num_points, d_point_offsets, d_mask, stream);
}

}  // extern "C"
