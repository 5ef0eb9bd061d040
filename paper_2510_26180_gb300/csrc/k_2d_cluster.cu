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
        for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
            const int lr = li / nx, ix = li - lr * nx;
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
                for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                    const int lr = li / nx, ix = li - lr * nx;
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
                    for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                        const int lr = li / nx, ix = li - lr * nx;
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
                        for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                            const int lr = li / nx, ix = li - lr * nx;
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
                    for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                        const int lr = li / nx, ix = li - lr * nx;
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
            for (int li = threadIdx.x; li < B.m; li += blockDim.x) {
                const int lr = li / nx, ix = li - lr * nx;
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
