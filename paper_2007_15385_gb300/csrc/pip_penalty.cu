// pip_penalty.cu -- differentiable collision penalty of a convex footprint
// placed at SE(2) poses, through the Voronoi margin:
//
//   L = sum_pose sum_point softplus(-m(x) / tau),   x = R(theta)^T (p - t),
//   m(x) = max_k (|x - p0|^2 - |x - p_k|^2) / (2 |p_k - p0|),
//
// the largest signed distance of x from the Voronoi edges (the bisectors of
// p0 and p_k, Eq. 2), with p0, p_k the footprint's centroid (Eq. 3-4) and
// mirrored generators (Eq. 8).  The gradient flows back through the edge
// that attains the max (lowest k among ties), through Eq. 8 and through
// Eq. 3-4 to the vertices, and through the rigid transform to the poses.
// Both calls rebuild the generator tables from the vertices (nothing is kept
// between forward and backward) inside a caller-provided workspace.
//
// Layout of the work: block (tile, pose) takes one pose and kPenPoints
// points; every thread keeps float32 partial sums (the backward pass's
// per-edge sums go through shared-memory atomics), the block reduces them in
// fp64 into its own slot of the workspace, and a final kernel adds the slots
// in a fixed order.
#include <stdlib.h>

#include "pip_prepare_kernel.cuh"

namespace {

constexpr int kPenThreads = 256;
constexpr int kPenPoints = 16384;  // points per block
constexpr int kPenMaxEdges = kMaxEdges;

struct PenWorkspace {
    PolyInfo *poly;
    int32_t *voffs;
    int32_t *worst;
    double2 *g0;
    double2 *gk;
    float4 *coef;
    float4 *coefn;
    double *loss_part;  // [blocks]
    double *pose_part;  // [blocks][3]  (sum g w_x, sum g w_y, sum g (w_x y - w_y x))
    double *edge_part;  // [blocks][n][3]  (sum g, sum g x, sum g y) per argmax edge
    double *edge_sum;   // [n][3]  reduced
    double *pose_sum;   // [P][3]  reduced
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t carve(void *base, int n, int P, int64_t blocks, PenWorkspace *w)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return (char *)base + o;
    };
    w->poly = (PolyInfo *)take(sizeof(PolyInfo));
    w->voffs = (int32_t *)take(2 * sizeof(int32_t));
    w->worst = (int32_t *)take(sizeof(int32_t));
    w->g0 = (double2 *)take(sizeof(double2));
    w->gk = (double2 *)take((size_t)n * sizeof(double2));
    w->coef = (float4 *)take((size_t)n * sizeof(float4));
    w->coefn = (float4 *)take((size_t)n * sizeof(float4));
    w->loss_part = (double *)take((size_t)blocks * sizeof(double));
    w->pose_part = (double *)take((size_t)blocks * 3 * sizeof(double));
    w->edge_part = (double *)take((size_t)blocks * n * 3 * sizeof(double));
    w->edge_sum = (double *)take((size_t)n * 3 * sizeof(double));
    w->pose_sum = (double *)take((size_t)P * 3 * sizeof(double));
    return off;
}

__global__ void pen_begin_kernel(int32_t *voffs, int32_t *worst, int n)
{
    if (threadIdx.x == 0) {
        voffs[0] = 0;
        voffs[1] = n;
        *worst = 0;
    }
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];  // fixed order
    return s;  // meaningful in thread 0
}

// softplus(z) = log(1 + e^z), evaluated without overflow
__device__ __forceinline__ float softplus_f(float z)
{
    return fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z)));
}

// sigmoid(z) = 1 / (1 + e^-z), evaluated without overflow
__device__ __forceinline__ float sigmoid_f(float z)
{
    const float e = __expf(-fabsf(z));
    return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}

template <bool BACKWARD>
__global__ void __launch_bounds__(kPenThreads) penalty_kernel(
    const PolyInfo *__restrict__ poly, const float4 *__restrict__ coefn, const float *__restrict__ poses,
    const float *__restrict__ pts, int64_t M, float tau, double *__restrict__ loss_part,
    double *__restrict__ pose_part, double *__restrict__ edge_part)
{
    __shared__ float4 cs[kPenMaxEdges];
    __shared__ float acc_edge[kPenMaxEdges][3];
    __shared__ double red[kPenThreads / 32];
    const PolyInfo pi = poly[0];
    const bool ok = pi.status == PIP_OK;
    const int n = ok ? pi.n : 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        cs[k] = coefn[k];
        acc_edge[k][0] = acc_edge[k][1] = acc_edge[k][2] = 0.f;
    }
    const int pose = blockIdx.y;
    const float tx = poses[3 * pose], ty = poses[3 * pose + 1], th = poses[3 * pose + 2];
    float sn, cn;
    sincosf(th, &sn, &cn);
    // x = R^T (p - t) - o = R^T (p - t'),  t' = t + R o
    const float tpx = tx + (cn * pi.ox - sn * pi.oy), tpy = ty + (sn * pi.ox + cn * pi.oy);
    const float inv_tau = 1.f / tau;
    __syncthreads();

    float l_acc = 0.f, a_x = 0.f, a_y = 0.f, a_t = 0.f;
    const int64_t p0 = (int64_t)blockIdx.x * kPenPoints;
    const int64_t p1 = min(p0 + kPenPoints, M);
    if (ok) {
        for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
            const float2 p = ((const float2 *)pts)[i];
            const float dx = p.x - tpx, dy = p.y - tpy;
            const float x = cn * dx + sn * dy;   // local body coordinates
            const float y = -sn * dx + cn * dy;
            float m = -INFINITY;
            int kb = 0;
            for (int k = 0; k < n; ++k) {
                const float4 c = cs[k];
                const float mk = fmaf(x, c.x, fmaf(y, c.y, -c.z));  // x . w/|w| - t/|w|
                if (BACKWARD) {
                    if (mk > m) { m = mk; kb = k; }
                } else {
                    m = fmaxf(m, mk);
                }
            }
            const float z = -m * inv_tau;
            if (!BACKWARD) {
                l_acc += softplus_f(z);
            } else {
                const float g = -sigmoid_f(z) * inv_tau;  // dL/dm
                if (g != 0.f) {
                    const float4 c = cs[kb];
                    const float xb = x + pi.ox, yb = y + pi.oy;  // body coordinates
                    a_x += g * c.x;
                    a_y += g * c.y;
                    a_t += g * (c.x * yb - c.y * xb);
                    atomicAdd(&acc_edge[kb][0], g);
                    atomicAdd(&acc_edge[kb][1], g * xb);
                    atomicAdd(&acc_edge[kb][2], g * yb);
                }
            }
        }
    }
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    if (!BACKWARD) {
        const double s = block_sum((double)l_acc, red);
        if (threadIdx.x == 0) loss_part[blk] = s;
    } else {
        const double sx = block_sum((double)a_x, red);
        if (threadIdx.x == 0) pose_part[3 * blk] = sx;
        const double sy = block_sum((double)a_y, red);
        if (threadIdx.x == 0) pose_part[3 * blk + 1] = sy;
        const double st = block_sum((double)a_t, red);
        if (threadIdx.x == 0) pose_part[3 * blk + 2] = st;
        __syncthreads();
        for (int e = threadIdx.x; e < 3 * pi.n; e += blockDim.x)
            edge_part[(size_t)blk * pi.n * 3 + e] = ok ? (double)acc_edge[e / 3][e % 3] : 0.0;
    }
}

// Fixed-order sums over the per-block slots.
__global__ void penalty_loss_reduce(const double *__restrict__ part, int64_t blocks,
                                    const float *__restrict__ grad_out, double *__restrict__ loss)
{
    __shared__ double red[kPenThreads / 32];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x) s += part[b];
    s = block_sum(s, red);
    if (threadIdx.x == 0) *loss = s;
    (void)grad_out;
}

// One block per reduced value, fixed order: values [0, 3n) are the edge sums
// over every block; values [3n, 3n + 3P) are pose j's sums over its tiles.
__global__ void __launch_bounds__(kPenThreads) penalty_backward_reduce(
    const double *__restrict__ edge_part, const double *__restrict__ pose_part, int n, int P,
    int64_t tiles, double *__restrict__ edge_sum, double *__restrict__ pose_sum)
{
    __shared__ double red[kPenThreads / 32];
    const int v = blockIdx.x;
    double s = 0.0;
    if (v < 3 * n) {
        const int64_t blocks = tiles * P;
        for (int64_t b = threadIdx.x; b < blocks; b += blockDim.x) s += edge_part[(size_t)b * 3 * n + v];
    } else {
        const int j = (v - 3 * n) / 3, c = (v - 3 * n) % 3;
        for (int64_t b = threadIdx.x; b < tiles; b += blockDim.x) s += pose_part[3 * ((int64_t)j * tiles + b) + c];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        if (v < 3 * n) edge_sum[v] = s;
        else pose_sum[v - 3 * n] = s;
    }
}

// Backward chain rule in fp64: one block, one thread per edge (n <= 64).
// Reduces the per-block slots, then
//   per edge k (N = |x - p0|^2 - |x - p_k|^2 summed affinely, D = |p_k - p0|):
//     dL/dp0  += -(X - S p0)/D + Nsum (p_k - p0) / (2 D^3)
//     dL/dp_k  =  (X - S p_k)/D - Nsum (p_k - p0) / (2 D^3)
//   then back through Eq. 8 (p_k = p0 - 2 L_k(p0) (a, b) / (a^2 + b^2)) and
//   Eq. 3-4 (p0 = C / (3 S2)) to the vertices; the pose gradients are
//   dL/dt = -R(theta) sum g w and dL/dtheta = sum g (w_x y - w_y x).
__global__ void __launch_bounds__(64) penalty_chain_kernel(
    const float *__restrict__ verts, int n, const double2 *__restrict__ g0tab,
    const double2 *__restrict__ gk, const PolyInfo *__restrict__ poly, const float *__restrict__ poses,
    int P, const double *__restrict__ pose_sum, const double *__restrict__ edge_sum,
    const float *__restrict__ grad_out, double *__restrict__ grad_v, double *__restrict__ grad_pose)
{
    __shared__ double sG0[2][64];
    __shared__ double sgv[64][2];
    const int k = threadIdx.x;
    const double scale = grad_out ? (double)grad_out[0] : 1.0;
    const bool ok = poly[0].status == PIP_OK;
    // pose gradients: one thread per pose, in a loop
    for (int j = k; j < P; j += blockDim.x) {
        const double ax = pose_sum[3 * j], ay = pose_sum[3 * j + 1], at = pose_sum[3 * j + 2];
        const double th = (double)poses[3 * j + 2];
        const double c = cos(th), s = sin(th);
        grad_pose[3 * j] = ok ? scale * -(c * ax - s * ay) : 0.0;
        grad_pose[3 * j + 1] = ok ? scale * -(s * ax + c * ay) : 0.0;
        grad_pose[3 * j + 2] = ok ? scale * at : 0.0;
    }
    double G0x = 0.0, G0y = 0.0;
    double gxm = 0.0, gym = 0.0, gxk = 0.0, gyk = 0.0;  // this edge's share of the vertex gradient
    const int km = k == 0 ? n - 1 : k - 1;
    if (ok && k < n) {
        const double S = edge_sum[3 * k], X = edge_sum[3 * k + 1], Y = edge_sum[3 * k + 2];
        const double2 g0 = g0tab[0], g = gk[k];
        const double ux = g.x - g0.x, uy = g.y - g0.y;
        const double D = sqrt(ux * ux + uy * uy);
        const double Nsum = 2.0 * (X * ux + Y * uy) + S * (g0.x * g0.x + g0.y * g0.y - g.x * g.x - g.y * g.y);
        const double D3 = 2.0 * D * D * D;
        const double Gkx = (X - S * g.x) / D - Nsum * ux / D3;
        const double Gky = (Y - S * g.y) / D - Nsum * uy / D3;
        G0x = -(X - S * g0.x) / D + Nsum * ux / D3;
        G0y = -(Y - S * g0.y) / D + Nsum * uy / D3;
        // Eq. 8 backward: a = y_k - y_{k-1}, b = x_{k-1} - x_k, c = x_k y_{k-1} - x_{k-1} y_k
        const double xm = verts[2 * km], ym = verts[2 * km + 1], xk = verts[2 * k], yk = verts[2 * k + 1];
        const double a = yk - ym, b = xm - xk, c = xk * ym - xm * yk;
        const double q = a * a + b * b;
        const double L = a * g0.x + b * g0.y + c;
        const double nG = a * Gkx + b * Gky;
        G0x += Gkx - 2.0 * a * nG / q;
        G0y += Gky - 2.0 * b * nG / q;
        // d p_k / d(a, b, c), contracted with G_k
        const double dA = -2.0 * (g0.x * nG / q + L * Gkx / q - 2.0 * a * L * nG / (q * q));
        const double dB = -2.0 * (g0.y * nG / q + L * Gky / q - 2.0 * b * L * nG / (q * q));
        const double dC = -2.0 * nG / q;
        // (a, b, c) as functions of v_{k-1} = (xm, ym) and v_k = (xk, yk)
        gxm = dB + dC * (-yk);
        gym = -dA + dC * xk;
        gxk = -dB + dC * ym;
        gyk = dA + dC * (-xm);
    }
    sG0[0][k] = G0x;
    sG0[1][k] = G0y;
    sgv[k][0] = 0.0;
    sgv[k][1] = 0.0;
    __syncthreads();
    // the vertex gradient from the generators: edge k touches v_{k-1} and v_k
    if (k < n) {
        atomicAdd(&sgv[km][0], gxm);
        atomicAdd(&sgv[km][1], gym);
        atomicAdd(&sgv[k][0], gxk);
        atomicAdd(&sgv[k][1], gyk);
    }
    __syncthreads();
    double Gx = 0.0, Gy = 0.0;
    for (int i = 0; i < n; ++i) {  // same order in every thread
        Gx += sG0[0][i];
        Gy += sG0[1][i];
    }
    // Eq. 3-4 backward: p0 = C / (3 S2), S2 = sum det_k, C = sum (v_{k-1} + v_k) det_k
    if (ok && k < n) {
        double S2 = 0.0;
        for (int i = 0; i < n; ++i) {
            const int im = i == 0 ? n - 1 : i - 1;
            S2 += (double)verts[2 * im] * verts[2 * i + 1] - (double)verts[2 * i] * verts[2 * im + 1];
        }
        const double2 g0 = g0tab[0];
        const double lx = Gx / (3.0 * S2), ly = Gy / (3.0 * S2);
        const double mu = -(Gx * g0.x + Gy * g0.y) / S2;
        const double xm = verts[2 * km], ym = verts[2 * km + 1], xk = verts[2 * k], yk = verts[2 * k + 1];
        const double det = xm * yk - xk * ym;
        const double sx = xm + xk, sy = ym + yk;
        // d det / d(xm, ym, xk, yk) = (yk, -xk, -ym, xm)
        atomicAdd(&sgv[km][0], lx * (det + sx * yk) + ly * (sy * yk) + mu * yk);
        atomicAdd(&sgv[km][1], lx * (sx * -xk) + ly * (det + sy * -xk) + mu * -xk);
        atomicAdd(&sgv[k][0], lx * (det + sx * -ym) + ly * (sy * -ym) + mu * -ym);
        atomicAdd(&sgv[k][1], lx * (sx * xm) + ly * (det + sy * xm) + mu * xm);
    }
    __syncthreads();
    if (k < n) {
        grad_v[2 * k] = ok ? scale * sgv[k][0] : 0.0;
        grad_v[2 * k + 1] = ok ? scale * sgv[k][1] : 0.0;
    }
}

pip_status check_args(const float *d_vertices, int32_t n, const float *d_poses, int32_t P,
                      const float *d_points, int64_t M, float tau, void *ws, size_t ws_bytes)
{
    if (d_vertices == nullptr || d_poses == nullptr || ws == nullptr) return PIP_E_INVALID_ARG;
    if (n < kMinEdges || n > kMaxEdges || P < 1 || M < 0 || !(tau > 0.f)) return PIP_E_INVALID_ARG;
    if (M > 0 && (d_points == nullptr || !aligned(d_points, 8))) return PIP_E_INVALID_ARG;
    if (!aligned(d_vertices, 8) || !aligned(d_poses, 4) || !aligned(ws, 256)) return PIP_E_INVALID_ARG;
    if (ws_bytes < pip_penalty_workspace_bytes(n, P, M)) return PIP_E_INVALID_ARG;
    return PIP_OK;
}

}  // namespace

extern "C" {

size_t pip_penalty_workspace_bytes(int32_t num_vertices, int32_t num_poses, int64_t num_points)
{
    if (num_vertices < 1 || num_poses < 1 || num_points < 0) return 0;
    const int64_t tiles = num_points > 0 ? (num_points + kPenPoints - 1) / kPenPoints : 1;
    PenWorkspace w;
    return carve(nullptr, num_vertices, num_poses, tiles * num_poses, &w) + 256;
}

pip_status pip_penalty_forward(const float *d_vertices, int32_t num_vertices, const float *d_poses,
                               int32_t num_poses, const float *d_points, int64_t num_points, float tau,
                               double *d_loss, void *d_workspace, size_t workspace_bytes, void *stream)
{
    pip_status st = check_args(d_vertices, num_vertices, d_poses, num_poses, d_points, num_points, tau,
                               d_workspace, workspace_bytes);
    if (st != PIP_OK) return st;
    if (d_loss == nullptr) return PIP_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tiles = num_points > 0 ? (num_points + kPenPoints - 1) / kPenPoints : 1;
    PenWorkspace w;
    carve(d_workspace, num_vertices, num_poses, tiles * num_poses, &w);
    pen_begin_kernel<<<1, 32, 0, s>>>(w.voffs, w.worst, num_vertices);
    prepare_kernel<<<1, 32, 0, s>>>(d_vertices, PIP_F32, w.voffs, 1, num_vertices, w.g0, w.gk, w.coef,
                                    w.coefn, w.poly, w.worst);
    penalty_kernel<false><<<dim3((unsigned)tiles, (unsigned)num_poses), kPenThreads, 0, s>>>(
        w.poly, w.coefn, d_poses, d_points, num_points, tau, w.loss_part, w.pose_part, w.edge_part);
    penalty_loss_reduce<<<1, kPenThreads, 0, s>>>(w.loss_part, tiles * num_poses, nullptr, d_loss);
    return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_E_CUDA;
}

pip_status pip_penalty_backward(const float *d_vertices, int32_t num_vertices, const float *d_poses,
                                int32_t num_poses, const float *d_points, int64_t num_points, float tau,
                                const float *d_grad_loss, double *d_grad_vertices, double *d_grad_poses,
                                void *d_workspace, size_t workspace_bytes, void *stream)
{
    pip_status st = check_args(d_vertices, num_vertices, d_poses, num_poses, d_points, num_points, tau,
                               d_workspace, workspace_bytes);
    if (st != PIP_OK) return st;
    if (d_grad_vertices == nullptr || d_grad_poses == nullptr) return PIP_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tiles = num_points > 0 ? (num_points + kPenPoints - 1) / kPenPoints : 1;
    PenWorkspace w;
    carve(d_workspace, num_vertices, num_poses, tiles * num_poses, &w);
    pen_begin_kernel<<<1, 32, 0, s>>>(w.voffs, w.worst, num_vertices);
    prepare_kernel<<<1, 32, 0, s>>>(d_vertices, PIP_F32, w.voffs, 1, num_vertices, w.g0, w.gk, w.coef,
                                    w.coefn, w.poly, w.worst);
    penalty_kernel<true><<<dim3((unsigned)tiles, (unsigned)num_poses), kPenThreads, 0, s>>>(
        w.poly, w.coefn, d_poses, d_points, num_points, tau, w.loss_part, w.pose_part, w.edge_part);
    penalty_backward_reduce<<<3 * num_vertices + 3 * num_poses, kPenThreads, 0, s>>>(
        w.edge_part, w.pose_part, num_vertices, num_poses, tiles, w.edge_sum, w.pose_sum);
    penalty_chain_kernel<<<1, 64, 0, s>>>(d_vertices, num_vertices, w.g0, w.gk, w.poly, d_poses, num_poses,
                                          w.pose_sum, w.edge_sum, d_grad_loss, d_grad_vertices,
                                          d_grad_poses);
    return cudaGetLastError() == cudaSuccess ? PIP_OK : PIP_E_CUDA;
}

}  // extern "C"
