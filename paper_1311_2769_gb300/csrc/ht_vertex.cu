// ht_vertex.cu — the second Hough transform: displaced vertices.
//
// Section "Displaced vertex identification": tracks from a common vertex
// (xv, yv) satisfy d0 = yv cos phi0 - xv sin phi0, so a second Hough
// transform of the first one's maxima finds the vertex.  Every candidate
// votes, with its cell's centre tables, for the (x, y) cells its line
// y cos phi - x sin phi = d0 crosses, walking the axis along which the line
// is less steep (one vote per bin of that axis, binary64 intrinsics in a
// fixed order, so the accumulator is reproducible bit for bit); vertices are
// the 2-D local maxima at or above a threshold by the first transform's
// linear-order tie rule (8-neighbourhood, no wrap), emitted in ascending
// (event, linear index) order.
#include <cuda_runtime.h>

#include <cstdint>

#include "ht_internal.h"

namespace ht {
namespace {

__device__ __forceinline__ int vbin(double u, double lo, double hi, int n) {
    const double t = __dmul_rn(__dsub_rn(u, lo), __ddiv_rn((double)n, __dsub_rn(hi, lo)));
    if (!(t >= 0.0 && t < (double)n)) return -1;
    return (int)t;
}

__global__ void vertex_vote_kernel(const VertexParams p) {
    int64_t np = *p.n_peaks;
    if (np > p.peak_cap) np = p.peak_cap;
    const int walk = max(p.nx, p.ny);
    const int64_t total = np * walk;
    const double xmin = p.xmin, xmax = p.xmax, ymin = p.ymin, ymax = p.ymax;
    const double wx = __ddiv_rn(__dsub_rn(xmax, xmin), (double)p.nx);
    const double wy = __ddiv_rn(__dsub_rn(ymax, ymin), (double)p.ny);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t pi = t / walk;
        const int u = (int)(t - pi * walk);
        const ht_peak pk = p.peaks[pi];
        if (pk.event < 0 || pk.event >= p.n_events) continue;
        const double cc = (double)p.cphi[pk.i_phi], ss = (double)p.sphi[pk.i_phi], dd = (double)p.d0[pk.i_d0].x;
        int a, b;
        if (fabs(cc) >= fabs(ss)) {
            if (u >= p.nx) continue;
            a = u;
            const double X = __dadd_rn(xmin, __dmul_rn(__dadd_rn((double)a, 0.5), wx));
            b = vbin(__ddiv_rn(__dadd_rn(dd, __dmul_rn(X, ss)), cc), ymin, ymax, p.ny);
        } else {
            if (u >= p.ny) continue;
            b = u;
            const double Y = __dadd_rn(ymin, __dmul_rn(__dadd_rn((double)b, 0.5), wy));
            a = vbin(__ddiv_rn(__dsub_rn(__dmul_rn(Y, cc), dd), ss), xmin, xmax, p.nx);
        }
        if (a < 0 || b < 0) continue;
        atomicAdd(p.acc + ((int64_t)pk.event * p.nx + a) * p.ny + b, 1u);
    }
}

// Is (a, b) of event row base `a1` a vertex?
__device__ __forceinline__ bool vertex_at(const VertexParams& p, const uint32_t* a1, int a, int b) {
    const int64_t self = (int64_t)a * p.ny + b;
    const uint32_t v = a1[self];
    if (v < p.thr) return false;
    for (int da = -1; da <= 1; ++da)
        for (int db = -1; db <= 1; ++db) {
            const int aa = a + da, bb = b + db;
            if ((da == 0 && db == 0) || aa < 0 || aa >= p.nx || bb < 0 || bb >= p.ny) continue;
            const int64_t other = (int64_t)aa * p.ny + bb;
            const uint32_t u = a1[other];
            if (other < self ? !(v > u) : !(v >= u)) return false;
        }
    return true;
}

// warp per (event, x row): EMIT = 0 counts the row's vertices, 1 writes them
template <bool EMIT>
__global__ void vertex_rows_kernel(const VertexParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t rows = (int64_t)p.n_events * p.nx;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += warps) {
        const int e = (int)(row / p.nx), a = (int)(row - (int64_t)e * p.nx);
        const uint32_t* a1 = p.acc + (int64_t)e * p.nx * p.ny;
        int64_t pos = EMIT ? p.rowbase[row] : 0;
        int n = 0;
        for (int b0 = 0; b0 < p.ny; b0 += 32) {
            const int b = b0 + lane;
            const bool is = b < p.ny && vertex_at(p, a1, a, b);
            const unsigned m = __ballot_sync(0xffffffffu, is);
            if (EMIT && is) {
                const int64_t q = pos + __popc(m & lt);
                if (q < p.cap) {
                    ht_vertex t;
                    t.event = e;
                    t.i_x = a;
                    t.i_y = b;
                    t.votes = a1[(int64_t)a * p.ny + b];
                    p.out[q] = t;
                }
            }
            pos += __popc(m);
            n += __popc(m);
        }
        if (!EMIT && lane == 0) p.rowcnt[row] = n;
    }
}

}  // namespace

cudaError_t launch_vertex_vote(const VertexParams& p, cudaStream_t s) {
    const int64_t work = p.peak_cap * (int64_t)(p.nx > p.ny ? p.nx : p.ny);
    if (work <= 0) return cudaSuccess;
    const int64_t want = (work + 255) / 256;
    const int grid = (int)(want < 152 * 32 ? want : 152 * 32);
    vertex_vote_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_vertex_rows(const VertexParams& p, bool emit, cudaStream_t s) {
    const int64_t rows = (int64_t)p.n_events * p.nx;
    if (rows <= 0) return cudaSuccess;
    const int64_t want = (rows * 32 + 255) / 256;
    const int grid = (int)(want < 152 * 16 ? want : 152 * 16);
    if (emit)
        vertex_rows_kernel<true><<<grid, 256, 0, s>>>(p);
    else
        vertex_rows_kernel<false><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ht
