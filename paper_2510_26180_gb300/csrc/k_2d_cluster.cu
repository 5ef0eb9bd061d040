// 2D systems too large for one CTA's shared memory, held in a thread-block
// cluster's distributed shared memory (mixed precision).
//
// The same propagator as k_fine2d_mixed (every backward-Euler step of
// (I + L_dt) v' = v + dt f0 solved by FP64 iterative refinement around an
// FP32 Jacobi-PCG, the FP64 residual test ||r||_2 <= rtol ||b||_2), for grids
// whose working set (FP32 weights, diagonal and five Krylov vectors, FP64
// solution and residual: ~48 B per unknown, 3.1 MB at 255^2) exceeds the
// 227 KB of one CTA.  A cluster of CL CTAs (one per SM) holds one system:
// CTA q owns the grid rows [q R, q R + R), R = ceil(nx / CL), with their
// weights and vector slices in its own shared memory.
//
// Across CTA boundaries only two things travel:
//   - the stencil's row above / below a CTA's block, read directly from the
//     neighbouring CTA's shared memory (distributed shared memory loads);
//   - the partial sums of the dot products: each CTA reduces its rows, writes
//     its partial, and after a cluster barrier every CTA adds the CL partials
//     in the same (rank) order, so all CTAs take the same, uniform
//     convergence decisions.
// The cluster barriers of the reductions also order every halo read after
// the neighbour's write of that vector and before its next overwrite (each
// vector is read across a boundary only in the pass after the one that
// wrote it, and a reduction separates any two passes); a barrier at the top
// of each work item orders the next item's overwrites after the previous
// item's last halo reads, and one at exit keeps every CTA's shared memory
// alive until no neighbour reads it.  Control flow is uniform over the
// cluster (same items, same decisions), so every barrier is reached by all
// of its threads.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace klecgc {

namespace {

constexpr int kThreadsCl = 512;
constexpr int kWarpsCl = kThreadsCl / 32;
constexpr int kMaxRefCl = 12;

// Sum of NV values over the cluster.  wred: [2][4][32] per-warp partials
// (this CTA), cpart: [2][4] this CTA's partials (read by every CTA of the
// cluster), cres: [2][4] the cluster sums.  ph alternates the halves.
template <int NV, typename T>
__device__ __forceinline__ void cluster_sum(T (&v)[NV], T* wred, T* cpart, T* cres, int& ph,
                                            const cg::cluster_group& cl) {
    static_assert(NV >= 1 && NV <= 4, "reduction width");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    T* b = wred + ph * 4 * 32;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) b[j * 32 + w] = v[j];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            T s = lane < kWarpsCl ? b[j * 32 + lane] : T(0);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) cpart[ph * 4 + j] = s;
        }
    }
    cl.sync();   // every CTA's partial written (release / acquire)
    const int ncl = (int)cl.num_blocks();
    if (w == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            T s = T(0);
            if (lane < ncl) s = cl.map_shared_rank(cpart, lane)[ph * 4 + j];
            // a fixed tree over the lanes: lane 0 adds in the same order in
            // every CTA, so all CTAs hold the same sum
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) cres[ph * 4 + j] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = cres[ph * 4 + j];
    ph ^= 1;
}

// Rows of this CTA's block and the neighbours' shared memory.
struct Block {
    int nx, R, r0, rows;       // R rows per CTA, this CTA's first row and row count
    int m;                     // rows * nx local unknowns
    const float* wx;           // [R][nx + 1] x-face weights of the local rows
    const float* wy;           // [R + 1][nx] y-faces r0 .. r0 + R (face f below row f)
    int has_s, has_n;          // a neighbour block exists below / above
};

// (c + sum_f w_f) v_i - sum_f w_f v_nb(f) on local unknown li (row lr, column
// ix) of the FP32 vector v; vs / vn: the rows below / above the block (the
// neighbours' last / first rows, in their shared memory).
__device__ __forceinline__ float stencil32(const Block& B, const float* v, const float* vs_row,
                                           const float* vn_row, int li, int lr, int ix, float c) {
    const int nx = B.nx;
    const float vi = v[li];
    const float* wr = B.wx + lr * (nx + 1) + ix;
    const float vw = ix > 0 ? v[li - 1] : 0.f;
    const float ve = ix < nx - 1 ? v[li + 1] : 0.f;
    const float vs = lr > 0 ? v[li - nx] : (B.has_s ? vs_row[ix] : 0.f);
    const float vn = lr < B.rows - 1 ? v[li + nx] : (B.has_n ? vn_row[ix] : 0.f);
    float acc = c * vi;
    acc = fmaf(wr[0], vi - vw, acc);
    acc = fmaf(wr[1], vi - ve, acc);
    acc = fmaf(B.wy[lr * nx + ix], vi - vs, acc);
    acc = fmaf(B.wy[(lr + 1) * nx + ix], vi - vn, acc);
    return acc;
}

// The FP64 operator (FP64 weights from global memory) on a local vector of
// type V (double: x; float: a correction d), neighbours' rows as above.
template <typename V>
__device__ __forceinline__ double stencil64(const Block& B, const double* wg, const V* v,
                                            const V* vs_row, const V* vn_row, int li, int lr,
                                            int ix, double c) {
    const int nx = B.nx, iy = B.r0 + lr;
    const double vi = (double)v[li];
    const double* wr = wg + (int64_t)iy * (nx + 1) + ix;
    const double* wyg = wg + (int64_t)nx * (nx + 1);
    const double vw = ix > 0 ? (double)v[li - 1] : 0.0;
    const double ve = ix < nx - 1 ? (double)v[li + 1] : 0.0;
    const double vs = lr > 0 ? (double)v[li - nx] : (B.has_s ? (double)vs_row[ix] : 0.0);
    const double vn = lr < B.rows - 1 ? (double)v[li + nx] : (B.has_n ? (double)vn_row[ix] : 0.0);
    double acc = c * vi;
    acc = fma(wr[0], vi - vw, acc);
    acc = fma(wr[1], vi - ve, acc);
    acc = fma(wyg[(int64_t)iy * nx + ix], vi - vs, acc);
    acc = fma(wyg[(int64_t)(iy + 1) * nx + ix], vi - vn, acc);
    return acc;
}

// A thread's walk over the local unknowns li = threadIdx.x, + blockDim.x, ...
// with their row and column kept by additions (an integer division by nx per
// unknown and pass cost more than the pass's arithmetic).
struct Walk {
    int li, lr, ix;
    int dl, dr, dc, nx;   // step in li, and the same as rows and columns
    __device__ __forceinline__ static Walk start(int nx) {
        Walk w;
        w.nx = nx;
        w.li = threadIdx.x;
        w.lr = threadIdx.x / nx;
        w.ix = threadIdx.x - w.lr * nx;
        w.dl = blockDim.x;
        w.dr = blockDim.x / nx;
        w.dc = blockDim.x - w.dr * nx;
        return w;
    }
    __device__ __forceinline__ void next(const Walk& w0) {
        li += w0.dl;
        lr += w0.dr;
        ix += w0.dc;
        if (ix >= w0.nx) {
            ix -= w0.nx;
            ++lr;
        }
    }
};

}  // namespace

// Shared memory per CTA: FP32 x-faces R (nx+1), y-faces (R+1) nx, diagonal
// and d, r, z, p, q (6 R nx); FP64 x and r (2 R nx).
size_t fine2d_cluster_smem(int nx, int CL) {
    const int R = (nx + CL - 1) / CL;
    const size_t m = (size_t)R * nx;
    const size_t f = (size_t)R * (nx + 1) + (size_t)(R + 1) * nx + 6 * m;
    return ((f * 4 + 15) & ~(size_t)15) + 2 * m * 8;
}

__global__ void __launch_bounds__(kThreadsCl) k_fine2d_mixed_cl(
    int64_t S, int N, int nx, int J, double dtc, double dtf, double alpha, int mode,
    const double* __restrict__ U, const double* __restrict__ u0, const double* __restrict__ wdt,
    double rtol2, float tin2, int maxit, double* __restrict__ out, const int* __restrict__ active,
    int* __restrict__ ifail, unsigned long long* __restrict__ itcount) {
    extern __shared__ __align__(16) unsigned char smc[];
    __shared__ double wred[2 * 4 * 32], cpart[2 * 4], cres[2 * 4];
    __shared__ float wred32[2 * 4 * 32], cpart32[2 * 4], cres32[2 * 4];
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int R = (nx + CL - 1) / CL;
    Block B;
    B.nx = nx;
    B.R = R;
    B.r0 = q * R;
    B.rows = max(0, min(R, nx - B.r0));
    B.m = B.rows * nx;
    B.has_s = q > 0 && B.rows > 0;
    B.has_n = B.r0 + B.rows < nx;
    const int mR = R * nx;
    float* wx = reinterpret_cast<float*>(smc);
    float* wy = wx + R * (nx + 1);
    float* dinv = wy + (R + 1) * nx;
    float* dv = dinv + mR;
    float* rv = dv + mR;
    float* zv = rv + mR;
    float* pv = zv + mR;
    float* qv = pv + mR;
    const size_t f = (size_t)R * (nx + 1) + (size_t)(R + 1) * nx + 6 * (size_t)mR;
    double* x = reinterpret_cast<double*>(smc + ((f * 4 + 15) & ~(size_t)15));
    double* r = x + mR;
    B.wx = wx;
    B.wy = wy;
    const Walk W0 = Walk::start(nx);
    // the neighbours' boundary rows: rank q-1's last row, rank q+1's first
    const int qs = q > 0 ? q - 1 : q, qn = q + 1 < CL ? q + 1 : q;
    const float* zs = cl.map_shared_rank(zv, qs) + (R - 1) * nx;
    const float* zn = cl.map_shared_rank(zv, qn);
    const float* ps = cl.map_shared_rank(pv, qs) + (R - 1) * nx;
    const float* pn = cl.map_shared_rank(pv, qn);
    const float* ds = cl.map_shared_rank(dv, qs) + (R - 1) * nx;
    const float* dn = cl.map_shared_rank(dv, qn);
    const double* xs = cl.map_shared_rank(x, qs) + (R - 1) * nx;
    const double* xn = cl.map_shared_rank(x, qn);

    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    const float c32 = (float)dtc;
    const int64_t items = mode == 0 ? S * N : S;
    const int64_t cid = blockIdx.x / CL, ncid = gridDim.x / CL;
    int ph = 0, ph32 = 0;
    unsigned long long its_total = 0;
    for (int64_t item = cid; item < items; item += ncid) {
        const int64_t s = mode == 0 ? item / N : item;
        const int n0 = mode == 0 ? (int)(item - s * N) : 0;
        if (!active[s]) continue;   // uniform over the cluster
        const double* wg = wdt + s * nf;
        cl.sync();   // the previous item's halo reads are done
        for (int e = threadIdx.x; e < B.rows * (nx + 1); e += blockDim.x)
            wx[e] = (float)wg[(int64_t)B.r0 * (nx + 1) + e];
        // faces r0 .. r0 + rows (a CTA without rows reads none: its r0 may
        // lie beyond the last face)
        for (int e = threadIdx.x; B.rows > 0 && e < (B.rows + 1) * nx; e += blockDim.x)
            wy[e] = (float)wg[(int64_t)nx * (nx + 1) + (int64_t)B.r0 * nx + e];
        __syncthreads();
        for (Walk c = W0; c.li < B.m; c.next(W0)) {
            const int li = c.li, lr = c.lr, ix = c.ix;
            const float* wr = wx + lr * (nx + 1) + ix;
            const float ws = wr[0] + wr[1] + wy[lr * nx + ix] + wy[(lr + 1) * nx + ix];
            dinv[li] = 1.f / (1.f + c32 + ws);
            const int i = B.r0 * nx + li;
            x[li] = (mode == 1 || n0 == 0) ? u0[i] : U[(s * n + i) * N + n0 - 1];
        }
        bool failed = false;
        const int nint = mode == 0 ? 1 : N;
        for (int ni = 0; ni < nint; ++ni) {
            for (int j = 0; j < J; ++j) {
                cl.sync();   // x complete in every CTA (its halo rows are read next)
                double v2[2] = {0.0, 0.0};   // ||b||^2, ||r||^2
                for (Walk c = W0; c.li < B.m; c.next(W0)) {
                    const int li = c.li, lr = c.lr, ix = c.ix;
                    const double ri = dtf - stencil64(B, wg, x, xs, xn, li, lr, ix, dtc);
                    const double bi = x[li] + dtf;
                    r[li] = ri;
                    v2[0] = fma(bi, bi, v2[0]);
                    v2[1] = fma(ri, ri, v2[1]);
                }
                cluster_sum<2>(v2, wred, cpart, cres, ph, cl);
                const double lim = rtol2 * v2[0];
                double rr64 = v2[1];
                int ref = 0;
                while (rr64 > lim) {
                    if (ref++ >= kMaxRefCl) {
                        failed = true;
                        break;
                    }
                    const double sigma = sqrt(rr64 / n), isig = 1.0 / sigma;
                    float w2[2] = {0.f, 0.f};   // r.z, ||r||^2
                    for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                        const float ri = (float)(r[li] * isig);
                        const float zi = dinv[li] * ri;
                        dv[li] = 0.f;
                        rv[li] = ri;
                        zv[li] = zi;
                        pv[li] = zi;
                        w2[0] = fmaf(ri, zi, w2[0]);
                        w2[1] = fmaf(ri, ri, w2[1]);
                    }
                    cluster_sum<2>(w2, wred32, cpart32, cres32, ph32, cl);
                    float rz = w2[0];
                    const float ilim = tin2 * w2[1];
                    float w1[1] = {0.f};
                    for (Walk c = W0; c.li < B.m; c.next(W0)) {
                        const int li = c.li, lr = c.lr, ix = c.ix;
                        const float qi = pv[li] + stencil32(B, pv, ps, pn, li, lr, ix, c32);
                        qv[li] = qi;
                        w1[0] = fmaf(pv[li], qi, w1[0]);
                    }
                    cluster_sum<1>(w1, wred32, cpart32, cres32, ph32, cl);
                    float pq = w1[0];
                    int it = 0;
                    for (;;) {
                        const float a = rz / pq;
                        float u2[2] = {0.f, 0.f};
                        for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                            dv[li] = fmaf(a, pv[li], dv[li]);
                            const float ri = fmaf(-a, qv[li], rv[li]);
                            const float zi = dinv[li] * ri;
                            rv[li] = ri;
                            zv[li] = zi;
                            u2[0] = fmaf(ri, ri, u2[0]);
                            u2[1] = fmaf(ri, zi, u2[1]);
                        }
                        cluster_sum<2>(u2, wred32, cpart32, cres32, ph32, cl);
                        ++it;
                        if (!(u2[0] > ilim) || it >= maxit) break;
                        const float rzn = u2[1];
                        const float beta = rzn / rz;
                        rz = rzn;
                        float y1[1] = {0.f};
                        for (Walk c = W0; c.li < B.m; c.next(W0)) {
                            const int li = c.li, lr = c.lr, ix = c.ix;
                            const float zi = zv[li];
                            const float pi = fmaf(beta, pv[li], zi);
                            const float qi =
                                fmaf(beta, qv[li], zi + stencil32(B, zv, zs, zn, li, lr, ix, c32));
                            pv[li] = pi;
                            qv[li] = qi;
                            y1[0] = fmaf(pi, qi, y1[0]);
                        }
                        cluster_sum<1>(y1, wred32, cpart32, cres32, ph32, cl);
                        pq = y1[0];
                    }
                    its_total += it;
                    // FP64 update: x += sigma d, r -= sigma (I + L) d
                    double z1[1] = {0.0};
                    for (Walk c = W0; c.li < B.m; c.next(W0)) {
                        const int li = c.li, lr = c.lr, ix = c.ix;
                        x[li] = fma(sigma, (double)dv[li], x[li]);
                        const double md = (double)dv[li] + stencil64(B, wg, dv, ds, dn, li, lr, ix, dtc);
                        const double ri = fma(-sigma, md, r[li]);
                        r[li] = ri;
                        z1[0] = fma(ri, ri, z1[0]);
                    }
                    cluster_sum<1>(z1, wred, cpart, cres, ph, cl);
                    rr64 = z1[0];
                }
            }
            if (mode == 1) {
                __syncthreads();
                for (int li = threadIdx.x; li < B.m; li += blockDim.x)
                    out[(s * n + B.r0 * nx + li) * N + ni] = x[li];
            }
        }
        if (mode == 0) {
            cl.sync();   // x complete in every CTA
            const double dTc = J * dtc;
            for (Walk c = W0; c.li < B.m; c.next(W0)) {
                const int li = c.li, lr = c.lr, ix = c.ix;
                const int i = B.r0 * nx + li;
                const double Fi = x[li];
                const double LF = J * (stencil64(B, wg, x, xs, xn, li, lr, ix, dtc) - dtc * Fi) + dTc * Fi;
                const double prev = n0 == 0 ? alpha * U[(s * n + i) * N + N - 1]
                                            : U[(s * n + i) * N + n0 - 1];
                out[(s * n + i) * N + n0] = (Fi + LF) - prev;
            }
        }
        if (failed && q == 0 && threadIdx.x == 0) ifail[s] = 1;
    }
    if (q == 0 && threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
    cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

// ------------------------------------------------------------------- CGC (b)
// The shifted solves (lambda_k I + L_dT) q = p of eq. three steps (b) on a
// cluster, as k_cgc_solve2d_mixed does them on one CTA: FP64 iterative
// refinement around FP32 Jacobi-COCG (unconjugated bilinear form; the matrix
// is complex symmetric), x accumulated in FP64 in the output p itself, the
// FP64 residual ||r||_2 <= rtol ||p_k||_2 as the stopping test.  Shared
// memory per CTA: FP32 weights and the complex FP32 vectors d, r, z, p, q of
// its rows; the FP64 complex residual (touched once per refinement, not per
// COCG iteration) in a global slice of its own, and the Jacobi diagonal
// recomputed where it is used (1 / (lambda + c + sum of the face weights)),
// which keeps a 255^2 system within 16 x 227 KB.
namespace {

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 jacobi_inv(const Block& B, int lr, int ix, float2 lc) {
    const int nx = B.nx;
    const float* wr = B.wx + lr * (nx + 1) + ix;
    const float dr = lc.x + wr[0] + wr[1] + B.wy[lr * nx + ix] + B.wy[(lr + 1) * nx + ix];
    const float di = lc.y;
    const float den = dr * dr + di * di;
    return make_float2(dr / den, -di / den);
}

// L32 (real weights, plus c) on a complex FP32 vector, neighbours' rows as
// in stencil32.
__device__ __forceinline__ float2 stencil32c(const Block& B, const float2* v, const float2* vs_row,
                                             const float2* vn_row, int li, int lr, int ix,
                                             float c) {
    const int nx = B.nx;
    const float2 z = make_float2(0.f, 0.f);
    const float2 vi = v[li];
    const float* wr = B.wx + lr * (nx + 1) + ix;
    const float2 vw = ix > 0 ? v[li - 1] : z;
    const float2 ve = ix < nx - 1 ? v[li + 1] : z;
    const float2 vs = lr > 0 ? v[li - nx] : (B.has_s ? vs_row[ix] : z);
    const float2 vn = lr < B.rows - 1 ? v[li + nx] : (B.has_n ? vn_row[ix] : z);
    const float a0 = wr[0], a1 = wr[1], a2 = B.wy[lr * nx + ix], a3 = B.wy[(lr + 1) * nx + ix];
    float re = c * vi.x, im = c * vi.y;
    re = fmaf(a0, vi.x - vw.x, re);
    im = fmaf(a0, vi.y - vw.y, im);
    re = fmaf(a1, vi.x - ve.x, re);
    im = fmaf(a1, vi.y - ve.y, im);
    re = fmaf(a2, vi.x - vs.x, re);
    im = fmaf(a2, vi.y - vs.y, im);
    re = fmaf(a3, vi.x - vn.x, re);
    im = fmaf(a3, vi.y - vn.y, im);
    return make_float2(re, im);
}

// (lambda I + L64) on the complex FP32 vector d, in FP64 (FP64 weights from
// global memory).
__device__ __forceinline__ double2 shift64c(const Block& B, const double* wg, const float2* d,
                                            const float2* ds_row, const float2* dn_row, int li,
                                            int lr, int ix, double c, double2 lk) {
    const int nx = B.nx, iy = B.r0 + lr;
    const float2 z = make_float2(0.f, 0.f);
    const float2 df = d[li];
    const double dr = df.x, di = df.y;
    const double* wr = wg + (int64_t)iy * (nx + 1) + ix;
    const double* wyg = wg + (int64_t)nx * (nx + 1);
    const float2 fw = ix > 0 ? d[li - 1] : z;
    const float2 fe = ix < nx - 1 ? d[li + 1] : z;
    const float2 fs = lr > 0 ? d[li - nx] : (B.has_s ? ds_row[ix] : z);
    const float2 fn = lr < B.rows - 1 ? d[li + nx] : (B.has_n ? dn_row[ix] : z);
    const double a0 = wr[0], a1 = wr[1], a2 = wyg[(int64_t)iy * nx + ix],
                 a3 = wyg[(int64_t)(iy + 1) * nx + ix];
    double re = fma(lk.x, dr, fma(-lk.y, di, c * dr));
    double im = fma(lk.x, di, fma(lk.y, dr, c * di));
    re = fma(a0, dr - fw.x, re);
    im = fma(a0, di - fw.y, im);
    re = fma(a1, dr - fe.x, re);
    im = fma(a1, di - fe.y, im);
    re = fma(a2, dr - fs.x, re);
    im = fma(a2, di - fs.y, im);
    re = fma(a3, dr - fn.x, re);
    im = fma(a3, di - fn.y, im);
    return make_double2(re, im);
}

}  // namespace

// Shared memory per CTA of the CGC layout: FP32 faces and five complex FP32
// vectors; global doubles per CTA: the complex FP64 residual of its rows.
size_t cgc2d_cluster_smem(int nx, int CL) {
    const int R = (nx + CL - 1) / CL;
    const size_t m = (size_t)R * nx;
    const size_t f = (size_t)R * (nx + 1) + (size_t)(R + 1) * nx;
    return ((f * 4 + 15) & ~(size_t)15) + 5 * m * 8;
}
int64_t cgc2d_cluster_scratch_per_cta(int nx, int CL) {
    const int R = (nx + CL - 1) / CL;
    return 2 * (int64_t)R * nx;
}

__global__ void __launch_bounds__(kThreadsCl) k_cgc_solve2d_mixed_cl(
    int64_t S, int K, int nx, double dTc, const double2* __restrict__ lam,
    const double* __restrict__ wdT, double rtol2, float tin2, int maxit,
    double2* __restrict__ pio, const int* __restrict__ active, int* __restrict__ ifail,
    unsigned long long* __restrict__ itcount, double* __restrict__ gscr) {
    extern __shared__ __align__(16) unsigned char smc[];
    __shared__ double wred[2 * 4 * 32], cpart[2 * 4], cres[2 * 4];
    __shared__ float wred32[2 * 4 * 32], cpart32[2 * 4], cres32[2 * 4];
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int R = (nx + CL - 1) / CL;
    Block B;
    B.nx = nx;
    B.R = R;
    B.r0 = q * R;
    B.rows = max(0, min(R, nx - B.r0));
    B.m = B.rows * nx;
    B.has_s = q > 0 && B.rows > 0;
    B.has_n = B.r0 + B.rows < nx;
    const int mR = R * nx;
    float* wx = reinterpret_cast<float*>(smc);
    float* wy = wx + R * (nx + 1);
    const size_t f = (size_t)R * (nx + 1) + (size_t)(R + 1) * nx;
    float2* dv = reinterpret_cast<float2*>(smc + ((f * 4 + 15) & ~(size_t)15));
    float2* rv = dv + mR;
    float2* zv = rv + mR;
    float2* pv = zv + mR;
    float2* qv = pv + mR;
    double2* r = reinterpret_cast<double2*>(gscr) + (int64_t)blockIdx.x * mR;
    B.wx = wx;
    B.wy = wy;
    const Walk W0 = Walk::start(nx);
    const int qs = q > 0 ? q - 1 : q, qn = q + 1 < CL ? q + 1 : q;
    const float2* zs = cl.map_shared_rank(zv, qs) + (R - 1) * nx;
    const float2* zn = cl.map_shared_rank(zv, qn);
    const float2* ps = cl.map_shared_rank(pv, qs) + (R - 1) * nx;
    const float2* pn = cl.map_shared_rank(pv, qn);
    const float2* ds = cl.map_shared_rank(dv, qs) + (R - 1) * nx;
    const float2* dn = cl.map_shared_rank(dv, qn);

    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    const float c32 = (float)dTc;
    const int64_t items = S * K;
    const int64_t cid = blockIdx.x / CL, ncid = gridDim.x / CL;
    int ph = 0, ph32 = 0;
    unsigned long long its_total = 0;
    for (int64_t item = cid; item < items; item += ncid) {
        const int64_t s = item / K;
        const int k = (int)(item - s * K);
        if (!active[s]) continue;   // uniform over the cluster
        const double* wg = wdT + s * nf;
        const double2 lk = lam[k];
        const float2 lk32 = make_float2((float)lk.x, (float)lk.y);
        const float2 lc = make_float2(lk32.x + c32, lk32.y);
        cl.sync();   // the previous item's halo reads are done
        for (int e = threadIdx.x; e < B.rows * (nx + 1); e += blockDim.x)
            wx[e] = (float)wg[(int64_t)B.r0 * (nx + 1) + e];
        for (int e = threadIdx.x; B.rows > 0 && e < (B.rows + 1) * nx; e += blockDim.x)
            wy[e] = (float)wg[(int64_t)nx * (nx + 1) + (int64_t)B.r0 * nx + e];
        double v1[1] = {0.0};   // ||b||^2
        for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
            double2* o = pio + (s * n + B.r0 * nx + li) * K + k;
            const double2 b = *o;
            r[li] = b;
            *o = make_double2(0.0, 0.0);   // x accumulates here
            v1[0] = fma(b.x, b.x, fma(b.y, b.y, v1[0]));
        }
        cluster_sum<1>(v1, wred, cpart, cres, ph, cl);   // (also orders the weights)
        const double lim = rtol2 * v1[0];
        double rr64 = v1[0];
        bool failed = false;
        int ref = 0;
        while (rr64 > lim) {
            if (ref++ >= kMaxRefCl) {
                failed = true;
                break;
            }
            const double sigma = sqrt(rr64 / n), isig = 1.0 / sigma;
            float v3[3] = {0.f, 0.f, 0.f};   // ||r||^2, r.z (complex, unconjugated)
            for (Walk c = W0; c.li < B.m; c.next(W0)) {
                const int li = c.li, lr = c.lr, ix = c.ix;
                const double2 rd = r[li];
                const float2 ri = make_float2((float)(rd.x * isig), (float)(rd.y * isig));
                const float2 zi = cmul2(jacobi_inv(B, lr, ix, lc), ri);
                dv[li] = make_float2(0.f, 0.f);
                rv[li] = ri;
                zv[li] = zi;
                pv[li] = zi;
                v3[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, v3[0]));
                v3[1] = fmaf(ri.x, zi.x, fmaf(-ri.y, zi.y, v3[1]));
                v3[2] = fmaf(ri.x, zi.y, fmaf(ri.y, zi.x, v3[2]));
            }
            cluster_sum<3>(v3, wred32, cpart32, cres32, ph32, cl);
            const float ilim = tin2 * v3[0];
            float rzr = v3[1], rzi = v3[2];
            float w2[2] = {0.f, 0.f};   // p.q with q = (lambda I + L) p
            for (Walk c = W0; c.li < B.m; c.next(W0)) {
                const int li = c.li, lr = c.lr, ix = c.ix;
                const float2 pi = pv[li];
                const float2 lp = stencil32c(B, pv, ps, pn, li, lr, ix, c32);
                const float2 qi = make_float2(lk32.x * pi.x - lk32.y * pi.y + lp.x,
                                              lk32.x * pi.y + lk32.y * pi.x + lp.y);
                qv[li] = qi;
                w2[0] = fmaf(pi.x, qi.x, fmaf(-pi.y, qi.y, w2[0]));
                w2[1] = fmaf(pi.x, qi.y, fmaf(pi.y, qi.x, w2[1]));
            }
            cluster_sum<2>(w2, wred32, cpart32, cres32, ph32, cl);
            float pqr = w2[0], pqi = w2[1];
            int it = 0;
            for (;;) {
                const float den = pqr * pqr + pqi * pqi;
                const float ar = (rzr * pqr + rzi * pqi) / den, ai = (rzi * pqr - rzr * pqi) / den;
                float u3[3] = {0.f, 0.f, 0.f};
                for (Walk c = W0; c.li < B.m; c.next(W0)) {
                    const int li = c.li, lr = c.lr, ix = c.ix;
                    const float2 pi = pv[li], qi = qv[li];
                    float2 di = dv[li], ri = rv[li];
                    di.x = fmaf(ar, pi.x, fmaf(-ai, pi.y, di.x));
                    di.y = fmaf(ar, pi.y, fmaf(ai, pi.x, di.y));
                    ri.x = fmaf(-ar, qi.x, fmaf(ai, qi.y, ri.x));
                    ri.y = fmaf(-ar, qi.y, fmaf(-ai, qi.x, ri.y));
                    const float2 zi = cmul2(jacobi_inv(B, lr, ix, lc), ri);
                    dv[li] = di;
                    rv[li] = ri;
                    zv[li] = zi;
                    u3[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, u3[0]));
                    u3[1] = fmaf(ri.x, zi.x, fmaf(-ri.y, zi.y, u3[1]));
                    u3[2] = fmaf(ri.x, zi.y, fmaf(ri.y, zi.x, u3[2]));
                }
                cluster_sum<3>(u3, wred32, cpart32, cres32, ph32, cl);
                ++it;
                if (!(u3[0] > ilim) || it >= maxit) break;
                const float dd = rzr * rzr + rzi * rzi;
                const float br = (u3[1] * rzr + u3[2] * rzi) / dd,
                            bi = (u3[2] * rzr - u3[1] * rzi) / dd;
                rzr = u3[1];
                rzi = u3[2];
                float y2[2] = {0.f, 0.f};
                for (Walk c = W0; c.li < B.m; c.next(W0)) {
                    const int li = c.li, lr = c.lr, ix = c.ix;
                    const float2 zi = zv[li], po = pv[li], qo = qv[li];
                    const float2 lz = stencil32c(B, zv, zs, zn, li, lr, ix, c32);
                    const float2 mz = make_float2(lk32.x * zi.x - lk32.y * zi.y + lz.x,
                                                  lk32.x * zi.y + lk32.y * zi.x + lz.y);
                    const float2 pnw = make_float2(fmaf(br, po.x, fmaf(-bi, po.y, zi.x)),
                                                   fmaf(br, po.y, fmaf(bi, po.x, zi.y)));
                    const float2 qnw = make_float2(fmaf(br, qo.x, fmaf(-bi, qo.y, mz.x)),
                                                   fmaf(br, qo.y, fmaf(bi, qo.x, mz.y)));
                    pv[li] = pnw;
                    qv[li] = qnw;
                    y2[0] = fmaf(pnw.x, qnw.x, fmaf(-pnw.y, qnw.y, y2[0]));
                    y2[1] = fmaf(pnw.x, qnw.y, fmaf(pnw.y, qnw.x, y2[1]));
                }
                cluster_sum<2>(y2, wred32, cpart32, cres32, ph32, cl);
                pqr = y2[0];
                pqi = y2[1];
            }
            its_total += it;
            // FP64 update: x += sigma d (in the output), r -= sigma (lambda I + L) d
            double z1[1] = {0.0};
            for (Walk c = W0; c.li < B.m; c.next(W0)) {
                const int li = c.li, lr = c.lr, ix = c.ix;
                double2* o = pio + (s * n + B.r0 * nx + li) * K + k;
                const float2 di = dv[li];
                double2 xo = *o;
                xo.x = fma(sigma, (double)di.x, xo.x);
                xo.y = fma(sigma, (double)di.y, xo.y);
                *o = xo;
                const double2 md = shift64c(B, wg, dv, ds, dn, li, lr, ix, dTc, lk);
                double2 ri = r[li];
                ri.x = fma(-sigma, md.x, ri.x);
                ri.y = fma(-sigma, md.y, ri.y);
                r[li] = ri;
                z1[0] = fma(ri.x, ri.x, fma(ri.y, ri.y, z1[0]));
            }
            cluster_sum<1>(z1, wred, cpart, cres, ph, cl);
            rr64 = z1[0];
        }
        if (failed && q == 0 && threadIdx.x == 0) ifail[s] = 1;
    }
    if (q == 0 && threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
    cl.sync();   // no CTA leaves while a neighbour may still read its shared memory
}

namespace {

template <typename K>
int cluster_plan(K kernel, int CL, size_t smem) {
    if (smem > (size_t)227 * 1024) return 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    if (CL > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kThreadsCl);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return ncl;
}

}  // namespace

// The largest cluster size that holds an nx x nx fine system (16, else 8),
// and the number of such clusters that fit on the GPU at once; 0 if none.
ClusterPlan2D fine2d_cluster_plan(int nx) {
    ClusterPlan2D p;
    for (int CL : {16, 8}) {
        const size_t smem = fine2d_cluster_smem(nx, CL);
        const int ncl = cluster_plan(k_fine2d_mixed_cl, CL, smem);
        if (ncl > 0) {
            p.CL = CL;
            p.clusters = ncl;
            p.smem = smem;
            return p;
        }
    }
    cudaGetLastError();
    return p;
}

ClusterPlan2D cgc2d_cluster_plan(int nx) {
    ClusterPlan2D p;
    for (int CL : {16, 8}) {
        const size_t smem = cgc2d_cluster_smem(nx, CL);
        const int ncl = cluster_plan(k_cgc_solve2d_mixed_cl, CL, smem);
        if (ncl > 0) {
            p.CL = CL;
            p.clusters = ncl;
            p.smem = smem;
            p.scratch_per_cta = cgc2d_cluster_scratch_per_cta(nx, CL);
            return p;
        }
    }
    cudaGetLastError();
    return p;
}

void launch_cgc_solve2d_mixed_cl(const ClusterPlan2D& p, int64_t S, int K, int nx, double dTc,
                                 const double2* lam, const double* wdT, double rtol, double tin,
                                 int maxit, Cplx<double>* pio, const int* active, int* ifail,
                                 unsigned long long* itcount, double* scratch, int64_t grid,
                                 cudaStream_t st) {
    if (S == 0 || p.CL == 0) return;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreadsCl);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = p.CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_cgc_solve2d_mixed_cl, S, K, nx, dTc, lam, wdT, rtol * rtol,
                       (float)(tin * tin), maxit, reinterpret_cast<double2*>(pio), active, ifail,
                       itcount, scratch);
}

void launch_fine2d_mixed_cl(const ClusterPlan2D& p, int64_t S, int N, int nx, int J, double dtc,
                            double dtf, double alpha, int mode, const double* U, const double* u0,
                            const double* wdt, double rtol, double tin, int maxit, double* out,
                            const int* active, int* ifail, unsigned long long* itcount,
                            cudaStream_t st) {
    if (S == 0 || p.CL == 0) return;
    const int64_t items = mode == 0 ? S * N : S;
    const int64_t ncl = std::min<int64_t>(p.clusters, items);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ncl * p.CL));
    cfg.blockDim = dim3(kThreadsCl);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = p.CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_fine2d_mixed_cl, S, N, nx, J, dtc, dtf, alpha, mode, U, u0, wdt,
                       rtol * rtol, (float)(tin * tin), maxit, out, active, ifail, itcount);
}

}  // namespace klecgc
