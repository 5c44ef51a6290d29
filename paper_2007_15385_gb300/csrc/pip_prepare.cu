// pip_prepare.cu -- polygon -> Voronoi generator tables (Sec. 3 of the paper),
// plus the lifecycle / status / export calls of the C ABI.
//
// One warp per polygon, lanes over edges (edge k = lane and lane + 32, n <= 64),
// fp64 throughout, warp-shuffle reductions.  Steps, in the paper's order:
//   1. Eq. 3 / Alg. 3: partial areas det_k = x_{k-1} y_k - x_k y_{k-1}, area.
//   2. Eq. 4 / Alg. 3: centroid p0 = sum (v_{k-1} + v_k) det_k / (6 A).
//   3. Alg. 4: a = y_k - y_{k-1}, b = x_{k-1} - x_k, c = -(a x_k + b y_k).
//   4. Eq. 8 / Alg. 4: p_k = (W p0 - 2 c (a, b)) / (a^2 + b^2).
//   5. The expanded Eq. 11 coefficients relative to o = float32(p0):
//        w_k = 2 (p_k - p0),  t_k = |p_k - o|^2 - |p0 - o|^2,
//      rounded to float32, and the error-bound scalars beta0, beta1.
// Vertices are first shifted by v_0 (translation leaves Eq. 4 and Eq. 8
// covariant) so that fp64 cancellation is relative to the polygon's own size.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pip_internal.cuh"

using namespace pip;

#include "pip_prepare_kernel.cuh"

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One warp per polygon: its coefficients at row j of a fixed-stride table,
// padded to a multiple of 4 edges with edges that never win the min
// (w = 0, t = +inf); an invalid polygon is one edge with t = -inf.
__global__ void pad_coef_kernel(const PolyInfo *__restrict__ poly, const float4 *__restrict__ coef, int P,
                                float4 *__restrict__ coefp)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (j >= P) return;
    const PolyInfo pi = poly[j];
    const bool ok = pi.status == PIP_OK;
    const int n = ok ? pi.n : 1;
    const int npad = (n + 3) & ~3;
    for (int k = lane; k < npad; k += 32) {
        float4 c;
        if (!ok) c = k == 0 ? make_float4(0.f, 0.f, -INFINITY, 0.f) : make_float4(0.f, 0.f, INFINITY, 0.f);
        else c = k < n ? coef[pi.voff + k] : make_float4(0.f, 0.f, INFINITY, 0.f);
        coefp[(size_t)j * kPadStride + k] = c;
    }
}

// One warp per float polygon: the comparators' rows.  Edge k joins
// u = v_{k-1} and v = v_k; dV = v - u and RHS = u_y dV_x - u_x dV_y in float32,
// as the listings form them (Alg. 1, Alg. 2), so that
// LHS - RHS = q_y dV_x - q_x dV_y - RHS is the two-FMA affine form the
// Voronoi kernels evaluate, t - x w_x - y w_y with (w_x, w_y, t) =
// (dV_y, -dV_x, -RHS).  Rows past n are NaN: the comparators' min and max
// ignore NaN, and a NaN edge is never in range.  Invalid polygons are
// skipped by their status.  The fp64 row holds the generators p_k and, in the
// last slot, p0.
__global__ void cmp_pad_kernel(const PolyInfo *__restrict__ poly, const float2 *__restrict__ verts,
                               const double2 *__restrict__ g0tab, const double2 *__restrict__ gktab, int P,
                               float4 *__restrict__ sign_rows, float4 *__restrict__ ray_rows,
                               double2 *__restrict__ g64_rows)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (j >= P) return;
    const PolyInfo pi = poly[j];
    const int n = pi.status == PIP_OK ? pi.n : 0;
    const float qnan = __int_as_float(0x7fc00000);
    for (int k = lane; k < kPadStride; k += 32) {
        float4 sg = make_float4(0.f, 0.f, qnan, 0.f);
        float4 r0 = make_float4(0.f, 0.f, qnan, 0.f), r1 = make_float4(qnan, qnan, 0.f, 0.f);
        double2 g = make_double2(0.0, 0.0);
        if (k < n) {
            const int km = k == 0 ? n - 1 : k - 1;
            const float2 u = verts[pi.voff + km], v = verts[pi.voff + k];
            const float dvx = v.x - u.x, dvy = v.y - u.y;
            const float rhs = fmaf(u.y, dvx, -(u.x * dvy));
            sg = make_float4(dvy, -dvx, -rhs, 0.f);
            const float s = v.y > u.y ? 1.f : -1.f;  // going up
            r0 = make_float4(s * dvy, -s * dvx, -s * rhs, 0.f);
            r1 = make_float4(u.y, v.y, 0.f, 0.f);
            g = gktab[pi.voff + k];
        }
        if (k == kPadStride - 1 && n > 0) g = g0tab[j];
        sign_rows[(size_t)j * kPadStride + k] = sg;
        ray_rows[(size_t)j * 2 * kPadStride + 2 * k] = r0;
        ray_rows[(size_t)j * 2 * kPadStride + 2 * k + 1] = r1;
        g64_rows[(size_t)j * kPadStride + k] = g;
    }
}

}  // namespace

namespace pip {

// pip_margin.cu: the pipelined margin kernel's shared-memory limit
cudaError_t margin_kernels_setup();

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

pip_status check_tables(const pip_tables *t)
{
    if (t == nullptr || t->base == nullptr) return PIP_E_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIP_E_CUDA;
    if (dev != t->device) return PIP_E_INVALID_ARG;
    return PIP_OK;
}

}  // namespace pip

extern "C" {

static pip_status prepare_impl(const void *d_vertices, pip_dtype vdtype, const int32_t *d_vertex_offsets,
                               int32_t num_polygons, int32_t total_vertices, int64_t max_points, int p0_kind,
                               const double *d_p0, void *stream, pip_tables **out);

pip_status pip_prepare(const void *d_vertices, pip_dtype vdtype, const int32_t *d_vertex_offsets,
                       int32_t num_polygons, int32_t total_vertices, int64_t max_points,
                       void *stream, pip_tables **out)
{
    return prepare_impl(d_vertices, vdtype, d_vertex_offsets, num_polygons, total_vertices, max_points,
                        kP0Centroid, nullptr, stream, out);
}

pip_status pip_prepare_p0(const void *d_vertices, pip_dtype vdtype, const int32_t *d_vertex_offsets,
                          int32_t num_polygons, int32_t total_vertices, int64_t max_points, int32_t p0_kind,
                          const double *d_p0, void *stream, pip_tables **out)
{
    if (p0_kind != PIP_P0_CENTROID && p0_kind != PIP_P0_VERTEX_MEAN && p0_kind != PIP_P0_GIVEN)
        return PIP_E_INVALID_ARG;
    if (p0_kind == PIP_P0_GIVEN && (d_p0 == nullptr || !aligned(d_p0, 16))) return PIP_E_INVALID_ARG;
    return prepare_impl(d_vertices, vdtype, d_vertex_offsets, num_polygons, total_vertices, max_points,
                        p0_kind, p0_kind == PIP_P0_GIVEN ? d_p0 : nullptr, stream, out);
}

static pip_status prepare_impl(const void *d_vertices, pip_dtype vdtype, const int32_t *d_vertex_offsets,
                               int32_t num_polygons, int32_t total_vertices, int64_t max_points, int p0_kind,
                               const double *d_p0, void *stream, pip_tables **out)
{
    if (out == nullptr) return PIP_E_INVALID_ARG;
    *out = nullptr;
    if (d_vertices == nullptr || d_vertex_offsets == nullptr) return PIP_E_INVALID_ARG;
    if (vdtype != PIP_F32 && vdtype != PIP_I32) return PIP_E_INVALID_ARG;
    if (num_polygons < 1 || total_vertices < 3) return PIP_E_INVALID_ARG;
    if ((int64_t)total_vertices > (int64_t)kMaxEdges * num_polygons) return PIP_E_INVALID_ARG;
    if (max_points < 0 || max_points > 0xFFFFFFFFll) return PIP_E_INVALID_ARG;
    if (!aligned(d_vertices, 8) || !aligned(d_vertex_offsets, 4)) return PIP_E_INVALID_ARG;

    pip_tables *t = (pip_tables *)calloc(1, sizeof(pip_tables));
    if (t == nullptr) return PIP_E_CUDA;
    if (cudaGetDevice(&t->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device) != cudaSuccess) {
        free(t);
        return PIP_E_CUDA;
    }
    t->P = num_polygons;
    t->V = total_vertices;
    t->vdtype = vdtype;
    t->capacity = max_points;

    const size_t P = (size_t)num_polygons, V = (size_t)total_vertices;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_verts = take(V * 8);
    const size_t o_voffs = take((P + 1) * 4);
    const size_t o_g0 = take(P * sizeof(double2));
    const size_t o_gk = take(V * sizeof(double2));
    const size_t o_coef = take(V * sizeof(float4));
    const size_t o_coefn = take(V * sizeof(float4));
    const size_t o_coefp = take(P * kPadStride * sizeof(float4));
    const size_t o_iedge = take(vdtype == PIP_I32 ? V * sizeof(int4) : 0);
    const size_t o_ipad = take(vdtype == PIP_I32 ? P * kPadStride * sizeof(int4) : 0);
    const size_t o_fpad = take(vdtype == PIP_I32 ? P * kPadStride * sizeof(float4) : 0);
    const size_t o_csign = take(vdtype == PIP_F32 ? P * kPadStride * sizeof(float4) : 0);
    const size_t o_cray = take(vdtype == PIP_F32 ? P * 2 * kPadStride * sizeof(float4) : 0);
    const size_t o_cg64 = take(vdtype == PIP_F32 ? P * kPadStride * sizeof(double2) : 0);
    const size_t o_poly = take(P * sizeof(PolyInfo));
    const size_t o_items = take((P + 1) * sizeof(int64_t));
    const size_t o_cnt = take(128);
    // refine queue: every point once, plus the slack of the pipelined kernel's
    // per-CTA slices (at most one tile of 4,096 points per CTA, 2 CTAs per SM)
    const size_t queue_entries = (size_t)max_points + (size_t)(t->num_sms + 1) * kStreamSlackPerSm;
    const size_t o_queue = take(queue_entries * sizeof(uint32_t));
    // all-pairs candidate keys (also used by one polygon when a first hit is asked for)
    const size_t o_keys = take((size_t)(max_points > 0 ? max_points : 1) * sizeof(uint32_t));
    t->bytes = off;
    if (cudaMalloc(&t->base, t->bytes) != cudaSuccess) {
        free(t);
        return PIP_E_CUDA;
    }
    char *b = (char *)t->base;
    t->d_verts = b + o_verts;
    t->d_voffs = (int32_t *)(b + o_voffs);
    t->d_g0 = (double2 *)(b + o_g0);
    t->d_gk = (double2 *)(b + o_gk);
    t->d_coef = (float4 *)(b + o_coef);
    t->d_coefn = (float4 *)(b + o_coefn);
    t->d_coefp = (float4 *)(b + o_coefp);
    t->d_iedge = vdtype == PIP_I32 ? (int4 *)(b + o_iedge) : nullptr;
    t->d_ipad = vdtype == PIP_I32 ? (int4 *)(b + o_ipad) : nullptr;
    t->d_fpad = vdtype == PIP_I32 ? (float4 *)(b + o_fpad) : nullptr;
    t->d_cmp_sign = vdtype == PIP_F32 ? (float4 *)(b + o_csign) : nullptr;
    t->d_cmp_ray = vdtype == PIP_F32 ? (float4 *)(b + o_cray) : nullptr;
    t->d_cmp_g64 = vdtype == PIP_F32 ? (double2 *)(b + o_cg64) : nullptr;
    t->d_poly = (PolyInfo *)(b + o_poly);
    t->d_items = (int64_t *)(b + o_items);
    t->d_qcount = (unsigned int *)(b + o_cnt);
    t->d_work = (unsigned int *)(b + o_cnt + 16);
    t->d_worst = (int32_t *)(b + o_cnt + 32);
    t->d_error = (int32_t *)(b + o_cnt + 48);
    t->d_stream_ctr = (void *)(b + o_cnt + 64);
    t->d_batch_ctr = (unsigned int *)(b + o_cnt + 96);
    t->d_queue = (uint32_t *)(b + o_queue);
    t->d_keys = (uint32_t *)(b + o_keys);

    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_verts, d_vertices, V * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(t->d_voffs, d_vertex_offsets, (P + 1) * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_cnt, 0, 128, s);
    if (e == cudaSuccess) e = stream_kernels_setup();
    if (e == cudaSuccess) e = margin_kernels_setup();
    if (e == cudaSuccess) e = allpairs_setup();
    if (e == cudaSuccess) e = ragged_kernels_setup();
    if (e == cudaSuccess) {
        const int threads = 256;
        const int blocks = (int)((P * 32 + threads - 1) / threads);
        prepare_kernel<<<blocks, threads, 0, s>>>(t->d_verts, vdtype, t->d_voffs, num_polygons,
                                                  total_vertices, t->d_g0, t->d_gk, t->d_coef,
                                                  t->d_coefn, t->d_poly, t->d_worst, p0_kind,
                                                  (const double2 *)d_p0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int threads = 256;
        const int blocks = (int)((P * 32 + threads - 1) / threads);
        pad_coef_kernel<<<blocks, threads, 0, s>>>(t->d_poly, t->d_coef, num_polygons, t->d_coefp);
        if (t->d_iedge) {
            int_edge_kernel<<<blocks, threads, 0, s>>>(t->d_poly, (const int2 *)t->d_verts, num_polygons,
                                                       t->d_iedge);
            int_pad_kernel<<<blocks, threads, 0, s>>>(t->d_poly, (const int2 *)t->d_verts, num_polygons,
                                                      t->d_ipad, t->d_fpad);
        } else {
            cmp_pad_kernel<<<blocks, threads, 0, s>>>(t->d_poly, (const float2 *)t->d_verts, t->d_g0, t->d_gk,
                                                      num_polygons, t->d_cmp_sign, t->d_cmp_ray, t->d_cmp_g64);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && num_polygons == 1) {
        // one polygon: keep its row and coefficients on the host too, so that
        // the pipelined kernel receives them as launch parameters
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMemcpy(&t->h_poly, t->d_poly, sizeof(PolyInfo), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) {
            const int n = total_vertices < kMaxEdges ? total_vertices : kMaxEdges;
            e = cudaMemcpy(t->h_coef, t->d_coef, (size_t)n * sizeof(float4), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && t->d_cmp_sign) {
                e = cudaMemcpy(t->h_cmp_sign, t->d_cmp_sign, (size_t)n * sizeof(float4), cudaMemcpyDeviceToHost);
                if (e == cudaSuccess)
                    e = cudaMemcpy(t->h_cmp_ray, t->d_cmp_ray, (size_t)2 * n * sizeof(float4),
                                   cudaMemcpyDeviceToHost);
            }
        }
        if (e == cudaSuccess) t->have_host_poly = 1;
    }
    if (e != cudaSuccess) {
        cudaFree(t->base);
        free(t);
        return PIP_E_CUDA;
    }
    *out = t;
    return PIP_OK;
}

void pip_destroy(pip_tables *t)
{
    if (t == nullptr) return;
    if (t->base) {
        cudaDeviceSynchronize();
        cudaFree(t->base);
    }
    if (t->events) {
        for (int i = 0; i < 3 * kTimingSlots; ++i) cudaEventDestroy(t->events[i]);
        free(t->events);
    }
    if (t->host_ready) {
        for (int i = 0; i < 65; ++i) cudaEventDestroy(t->host_events[i]);
        cudaStreamDestroy(t->host_copy_stream);
    }
    free(t);
}

pip_status pip_timing(pip_tables *t, int enable)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (enable && t->events == nullptr) {
        cudaEvent_t *ev = (cudaEvent_t *)calloc(3 * kTimingSlots, sizeof(cudaEvent_t));
        if (ev == nullptr) return PIP_E_CUDA;
        for (int i = 0; i < 3 * kTimingSlots; ++i) {
            if (cudaEventCreate(&ev[i]) != cudaSuccess) {
                for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
                free(ev);
                return PIP_E_CUDA;
            }
        }
        t->events = ev;
    }
    t->timing = enable ? 1 : 0;
    t->timed_calls = 0;
    return PIP_OK;
}

pip_status pip_timing_read(pip_tables *t, int32_t *calls, double *bulk_ms, double *refine_ms)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    double b = 0.0, r = 0.0;
    const int n = t->timed_calls < kTimingSlots ? t->timed_calls : kTimingSlots;
    for (int i = 0; i < n && t->events; ++i) {
        float ms1 = 0.f, ms2 = 0.f;
        PIP_CUDA_TRY(cudaEventSynchronize(t->events[3 * i + 2]));
        PIP_CUDA_TRY(cudaEventElapsedTime(&ms1, t->events[3 * i], t->events[3 * i + 1]));
        PIP_CUDA_TRY(cudaEventElapsedTime(&ms2, t->events[3 * i + 1], t->events[3 * i + 2]));
        b += ms1;
        r += ms2;
    }
    if (calls) *calls = n;
    if (bulk_ms) *bulk_ms = b;
    if (refine_ms) *refine_ms = r;
    t->timed_calls = 0;
    return PIP_OK;
}

int32_t pip_num_polygons(const pip_tables *t) { return t ? t->P : 0; }
int32_t pip_total_vertices(const pip_tables *t) { return t ? t->V : 0; }

pip_status pip_get_status(const pip_tables *t, void *stream, int64_t *refine_count)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    PIP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int32_t worst = 0, error = 0;
    unsigned int cnt = 0;
    PIP_CUDA_TRY(cudaMemcpy(&error, t->d_error, sizeof(error), cudaMemcpyDeviceToHost));
    if (error != 0) {
        PIP_CUDA_TRY(cudaMemset(t->d_error, 0, sizeof(int32_t)));
        if (refine_count) *refine_count = 0;
        return (pip_status)error;
    }
    PIP_CUDA_TRY(cudaMemcpy(&worst, t->d_worst, sizeof(worst), cudaMemcpyDeviceToHost));
    PIP_CUDA_TRY(cudaMemcpy(&cnt, t->d_qcount, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (refine_count) *refine_count = (int64_t)cnt;
    return (pip_status)worst;
}

pip_status pip_get_polygon_status(const pip_tables *t, int32_t *h_status, void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    if (h_status == nullptr) return PIP_E_INVALID_ARG;
    PIP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    for (int j = 0; j < t->P; ++j) {
        PIP_CUDA_TRY(cudaMemcpy(&h_status[j], &t->d_poly[j].status, sizeof(int32_t),
                                cudaMemcpyDeviceToHost));
    }
    return PIP_OK;
}

pip_status pip_export_tables(const pip_tables *t, double *h_g0, double *h_gk, float *h_coef,
                             float *h_origin, float *h_bound, float *h_disc, void *stream)
{
    pip_status st = check_tables(t);
    if (st != PIP_OK) return st;
    PIP_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    const size_t P = (size_t)t->P, V = (size_t)t->V;
    if (h_g0) PIP_CUDA_TRY(cudaMemcpy(h_g0, t->d_g0, P * sizeof(double2), cudaMemcpyDeviceToHost));
    if (h_gk) PIP_CUDA_TRY(cudaMemcpy(h_gk, t->d_gk, V * sizeof(double2), cudaMemcpyDeviceToHost));
    if (h_coef) PIP_CUDA_TRY(cudaMemcpy(h_coef, t->d_coef, V * sizeof(float4), cudaMemcpyDeviceToHost));
    if (h_origin || h_bound || h_disc) {
        PolyInfo *tmp = (PolyInfo *)malloc(P * sizeof(PolyInfo));
        if (tmp == nullptr) return PIP_E_CUDA;
        if (cudaMemcpy(tmp, t->d_poly, P * sizeof(PolyInfo), cudaMemcpyDeviceToHost) != cudaSuccess) {
            free(tmp);
            return PIP_E_CUDA;
        }
        for (size_t j = 0; j < P; ++j) {
            if (h_origin) { h_origin[2 * j] = tmp[j].ox; h_origin[2 * j + 1] = tmp[j].oy; }
            if (h_bound) { h_bound[2 * j] = tmp[j].beta0; h_bound[2 * j + 1] = tmp[j].beta1; }
            if (h_disc) { h_disc[2 * j] = tmp[j].tin; h_disc[2 * j + 1] = tmp[j].tout; }
        }
        free(tmp);
    }
    return PIP_OK;
}

const char *pip_status_string(pip_status s)
{
    switch (s) {
    case PIP_OK: return "ok";
    case PIP_E_INVALID_ARG: return "invalid argument";
    case PIP_E_DEGENERATE: return "degenerate polygon (repeated vertex, zero area or centroid not interior)";
    case PIP_E_NONCONVEX: return "non-convex polygon";
    case PIP_E_NONFINITE: return "non-finite vertex coordinate";
    case PIP_E_CUDA: return "CUDA runtime error";
    case PIP_E_TIMEOUT: return "device-side wait timed out";
    case PIP_E_CAPACITY: return "more points than the prepared capacity";
    }
    return "unknown status";
}

}  // extern "C"
