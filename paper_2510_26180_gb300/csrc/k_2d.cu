// 2D problem (five-point operator on an nx x nx interior grid): the fine
// propagator F (with the CGC right-hand side as its epilogue) and the shifted
// CGC solves of eq. three steps (b), both by preconditioned Krylov
// iterations, one CTA per linear system.
//
// Operator (flux form, zero Dirichlet values, unknown (ix, iy) at index
// i = iy*nx + ix):  (L v)_i = c' v_i + sum_f w_f (v_i - v_nb(f))
// over the four faces f of cell i; a neighbour outside the grid is 0.
// Per sample the face weights are stored x-faces first, then y-faces:
//   wx[iy][fx], fx = 0..nx (face between ix = fx-1 and ix = fx),
//   wy[fy][ix], fy = 0..nx (face between iy = fy-1 and iy = fy),
// scaled by the step: w = dt a / h^2 for F, w = dT a / h^2 for the CGC,
// with c' = dt c or dT c accordingly.
//
//  F:   (I + L_dt) v^{m+1} = v^m + dt f0, J steps, Jacobi-preconditioned CG
//       warm-started from v^m, stopped at ||r||_2 <= rtol ||b||_2.
//  CGC: (lambda_k I + L_dT) q_k = p_k, Jacobi-preconditioned COCG (CG with the
//       unconjugated bilinear form; lambda_k I + L is complex symmetric),
//       stopped at ||r||_2 <= rtol ||p_k||_2.
//
// Advection-diffusion (b = b0 (x2, x1) >= 0, upwind): L gains
//   adv (iy+1) (v_i - v_W) + adv (ix+1) (v_i - v_S),  adv = dt b0 or dT b0,
// the operator is no longer symmetric, and both solves use Jacobi-
// preconditioned BiCGStab (right preconditioning; Hermitian inner products
// in the complex case) instead of CG / COCG, with the same stopping rules.
//
// Each CTA keeps its system's weights, diagonal and Krylov vectors in shared
// memory when they fit (else in a global slice of its own) and loops over
// work items.  The mixed-precision systems that do not fit one CTA go to the
// thread-block-cluster kernels of k_2d_cluster.cu instead (plan_2d).  The two dot products of an iteration are fused into two block
// reductions; every thread sums the per-warp partials in the same order, so
// all threads take the same (uniform) convergence decision.  Iteration
// counts are capped (maxit); a solve that reaches the cap sets ifail[s].
#include "common.cuh"

namespace klecgc {

namespace {

constexpr int kThreads2d = 256;
constexpr int kWarps2d = kThreads2d / 32;

// Sum of NV <= 3 values over the block; red: [2][3][32] doubles, ph alternates.
// The two halves are fixed (stride 3 x 32 whatever NV is), so consecutive
// reductions never share a slot: a warp that races ahead into the next
// reduction writes the other half while slower warps still read this one.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red, int& ph) {
    static_assert(NV >= 1 && NV <= 3, "reduction width");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    double* b = red + ph * 3 * 32;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) b[j * 32 + w] = v[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double s = 0.0;
        for (int q = 0; q < kWarps2d; ++q) s += b[j * 32 + q];
        v[j] = s;
    }
    ph ^= 1;
}

// The same reduction in FP32 (the inner solves of the mixed propagator; FP64
// adds run at 1/64 of the FP32 rate).  red32: [2][3][32] floats.
template <int NV>
__device__ __forceinline__ void block_sum32(float (&v)[NV], float* red32, int& ph) {
    static_assert(NV >= 1 && NV <= 3, "reduction width");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    float* b = red32 + ph * 3 * 32;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) b[j * 32 + w] = v[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        float s = 0.f;
        for (int q = 0; q < kWarps2d; ++q) s += b[j * 32 + q];
        v[j] = s;
    }
    ph ^= 1;
}

// sum over the four faces of w_f (v_i - v_nb), plus c' v_i.
struct Stencil {
    const double* wx;
    const double* wy;
    int nx;
    __device__ __forceinline__ double apply(const double* v, int i, int ix, int iy, double c) const {
        const double vi = v[i];
        const double* wr = wx + iy * (nx + 1) + ix;
        const double vw = ix > 0 ? v[i - 1] : 0.0;
        const double ve = ix < nx - 1 ? v[i + 1] : 0.0;
        const double vs = iy > 0 ? v[i - nx] : 0.0;
        const double vn = iy < nx - 1 ? v[i + nx] : 0.0;
        double acc = c * vi;
        acc = fma(wr[0], vi - vw, acc);
        acc = fma(wr[1], vi - ve, acc);
        acc = fma(wy[iy * nx + ix], vi - vs, acc);
        acc = fma(wy[(iy + 1) * nx + ix], vi - vn, acc);
        return acc;
    }
    __device__ __forceinline__ double2 apply2(const double2* v, int i, int ix, int iy, double c) const {
        const double2 vi = v[i];
        const double2 z = make_double2(0.0, 0.0);
        const double* wr = wx + iy * (nx + 1) + ix;
        const double2 vw = ix > 0 ? v[i - 1] : z;
        const double2 ve = ix < nx - 1 ? v[i + 1] : z;
        const double2 vs = iy > 0 ? v[i - nx] : z;
        const double2 vn = iy < nx - 1 ? v[i + nx] : z;
        const double a0 = wr[0], a1 = wr[1], a2 = wy[iy * nx + ix], a3 = wy[(iy + 1) * nx + ix];
        double re = c * vi.x, im = c * vi.y;
        re = fma(a0, vi.x - vw.x, re);
        im = fma(a0, vi.y - vw.y, im);
        re = fma(a1, vi.x - ve.x, re);
        im = fma(a1, vi.y - ve.y, im);
        re = fma(a2, vi.x - vs.x, re);
        im = fma(a2, vi.y - vs.y, im);
        re = fma(a3, vi.x - vn.x, re);
        im = fma(a3, vi.y - vn.y, im);
        return make_double2(re, im);
    }
    // sum of the four face weights of cell i
    __device__ __forceinline__ double wsum(int ix, int iy) const {
        const double* wr = wx + iy * (nx + 1) + ix;
        return wr[0] + wr[1] + wy[iy * nx + ix] + wy[(iy + 1) * nx + ix];
    }
};

__device__ __forceinline__ void cpy_weights(double* dst, const double* src, int nf) {
    for (int e = threadIdx.x; e < nf; e += blockDim.x) dst[e] = src[e];
}

// ------------------------------------------------------------------- F
// mode 0 (parareal sweep): item (s, n); start = u0 (n = 0) or U[s][.][n-1];
//   after J steps writes r[s][i][n] = (I + L_dT) F_i - prev_i with
//   prev = alpha U[s][.][N-1] (n = 0) or U[s][.][n-1]; L_dT = J L_dt.
// mode 1 (sequential fine solution): item s; start u0; after every J steps
//   writes out[s][i][n] = v_i.
// U, out: internal layout [S][n_unknowns][N].
__global__ void __launch_bounds__(kThreads2d) k_fine2d(
    int64_t S, int N, int nx, int J, double dtc, double dtf, double alpha, int mode,
    const double* __restrict__ U, const double* __restrict__ u0, const double* __restrict__ wdt,
    double rtol2, int maxit, double* __restrict__ out, const int* __restrict__ active,
    int* __restrict__ ifail, unsigned long long* __restrict__ itcount, double* __restrict__ gscr,
    int64_t per_cta) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red[2 * 3 * 32];
    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    double* W = gscr ? gscr + blockIdx.x * per_cta : dsm;
    double* dinv = W + nf;
    double* x = dinv + n;
    double* r = x + n;
    double* z = r + n;
    double* p = z + n;
    double* q = p + n;
    const Stencil L{W, W + nx * (nx + 1), nx};
    const int64_t items = mode == 0 ? S * N : S;
    int ph = 0;
    unsigned long long its_total = 0;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t s = mode == 0 ? item / N : item;
        const int n0 = mode == 0 ? (int)(item - s * N) : 0;
        if (!active[s]) continue;
        __syncthreads();  // the previous item's epilogue has read its vectors
        cpy_weights(W, wdt + s * nf, nf);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int iy = i / nx, ix = i - iy * nx;
            dinv[i] = 1.0 / (1.0 + dtc + L.wsum(ix, iy));
            x[i] = (mode == 1 || n0 == 0) ? u0[i] : U[(s * n + i) * N + n0 - 1];
        }
        bool failed = false;
        const int nint = mode == 0 ? 1 : N;
        for (int ni = 0; ni < nint; ++ni) {
            for (int j = 0; j < J; ++j) {
                __syncthreads();  // x complete
                // r = b - M x = dtf - L x, z = D^{-1} r, p = z
                double v3[3] = {0.0, 0.0, 0.0};  // ||b||^2, r.z, ||r||^2
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double xi = x[i];
                    const double ri = dtf - L.apply(x, i, ix, iy, dtc);
                    const double zi = dinv[i] * ri;
                    r[i] = ri;
                    z[i] = zi;
                    p[i] = zi;
                    const double bi = xi + dtf;
                    v3[0] = fma(bi, bi, v3[0]);
                    v3[1] = fma(ri, zi, v3[1]);
                    v3[2] = fma(ri, ri, v3[2]);
                }
                block_sum<3>(v3, red, ph);
                const double lim = rtol2 * v3[0];
                double rz = v3[1];
                if (!(v3[2] > lim)) continue;  // x already solves the step
                // q = M p, p.q
                double v1[1] = {0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double qi = p[i] + L.apply(p, i, ix, iy, dtc);
                    q[i] = qi;
                    v1[0] = fma(p[i], qi, v1[0]);
                }
                block_sum<1>(v1, red, ph);
                double pq = v1[0];
                int it = 0;
                for (;;) {
                    const double a = rz / pq;
                    double v2[2] = {0.0, 0.0};  // ||r||^2, r.z
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        x[i] = fma(a, p[i], x[i]);
                        const double ri = fma(-a, q[i], r[i]);
                        const double zi = dinv[i] * ri;
                        r[i] = ri;
                        z[i] = zi;
                        v2[0] = fma(ri, ri, v2[0]);
                        v2[1] = fma(ri, zi, v2[1]);
                    }
                    block_sum<2>(v2, red, ph);
                    ++it;
                    if (!(v2[0] > lim)) break;
                    if (it >= maxit) {
                        failed = true;
                        break;
                    }
                    const double beta = v2[1] / rz;
                    rz = v2[1];
                    // p = z + beta p, q = M z + beta q (= M p)
                    double w1[1] = {0.0};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const int iy = i / nx, ix = i - iy * nx;
                        const double zi = z[i];
                        const double pi = fma(beta, p[i], zi);
                        const double qi = fma(beta, q[i], zi + L.apply(z, i, ix, iy, dtc));
                        p[i] = pi;
                        q[i] = qi;
                        w1[0] = fma(pi, qi, w1[0]);
                    }
                    block_sum<1>(w1, red, ph);
                    pq = w1[0];
                }
                its_total += it;
            }
            if (mode == 1) {
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) out[(s * n + i) * N + ni] = x[i];
            }
        }
        if (mode == 0) {
            __syncthreads();  // x complete
            const double dTc = J * dtc;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int iy = i / nx, ix = i - iy * nx;
                const double Fi = x[i];
                const double LF = J * (L.apply(x, i, ix, iy, dtc) - dtc * Fi) + dTc * Fi;
                const double prev = n0 == 0 ? alpha * U[(s * n + i) * N + N - 1]
                                            : U[(s * n + i) * N + n0 - 1];
                out[(s * n + i) * N + n0] = (Fi + LF) - prev;
            }
        }
        if (failed && threadIdx.x == 0) ifail[s] = 1;
    }
    if (threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
}

// The five-point operator plus the upwind convection (advection-diffusion).
struct StencilAdv {
    Stencil L;
    double adv;   // step * b0
    __device__ __forceinline__ double apply(const double* v, int i, int ix, int iy, double c) const {
        const double vi = v[i];
        const double vw = ix > 0 ? v[i - 1] : 0.0;
        const double vs = iy > 0 ? v[i - L.nx] : 0.0;
        double acc = L.apply(v, i, ix, iy, c);
        acc = fma(adv * (iy + 1), vi - vw, acc);
        acc = fma(adv * (ix + 1), vi - vs, acc);
        return acc;
    }
    __device__ __forceinline__ double2 apply2(const double2* v, int i, int ix, int iy,
                                              double c) const {
        const double2 vi = v[i];
        const double2 z = make_double2(0.0, 0.0);
        const double2 vw = ix > 0 ? v[i - 1] : z;
        const double2 vs = iy > 0 ? v[i - L.nx] : z;
        double2 acc = L.apply2(v, i, ix, iy, c);
        const double a1 = adv * (iy + 1), a2 = adv * (ix + 1);
        acc.x = fma(a1, vi.x - vw.x, acc.x);
        acc.y = fma(a1, vi.y - vw.y, acc.y);
        acc.x = fma(a2, vi.x - vs.x, acc.x);
        acc.y = fma(a2, vi.y - vs.y, acc.y);
        return acc;
    }
    __device__ __forceinline__ double diag(int ix, int iy) const {
        return L.wsum(ix, iy) + adv * (iy + 1) + adv * (ix + 1);
    }
};

// ------------------------------------------------------------------- F, advection
// k_fine2d with BiCGStab for the non-symmetric backward-Euler systems
// (I + L_dt) v' = v + dt f0, warm-started from v; modes and outputs as
// k_fine2d.  adv = dt b0.  Working storage: weights, dinv, x, r (also s),
// rh, p, v, y (also z), t.
__global__ void __launch_bounds__(kThreads2d) k_fine2d_bicgs(
    int64_t S, int N, int nx, int J, double dtc, double dtf, double adv, double alpha, int mode,
    const double* __restrict__ U, const double* __restrict__ u0, const double* __restrict__ wdt,
    double rtol2, int maxit, double* __restrict__ out, const int* __restrict__ active,
    int* __restrict__ ifail, unsigned long long* __restrict__ itcount, double* __restrict__ gscr,
    int64_t per_cta) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red[2 * 3 * 32];
    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    double* W = gscr ? gscr + blockIdx.x * per_cta : dsm;
    double* dinv = W + nf;
    double* x = dinv + n;
    double* r = x + n;
    double* rh = r + n;
    double* p = rh + n;
    double* v = p + n;
    double* y = v + n;
    double* t = y + n;
    const StencilAdv L{{W, W + nx * (nx + 1), nx}, adv};
    const int64_t items = mode == 0 ? S * N : S;
    int ph = 0;
    unsigned long long its_total = 0;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t s = mode == 0 ? item / N : item;
        const int n0 = mode == 0 ? (int)(item - s * N) : 0;
        if (!active[s]) continue;
        __syncthreads();  // the previous item's epilogue has read its vectors
        cpy_weights(W, wdt + s * nf, nf);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int iy = i / nx, ix = i - iy * nx;
            dinv[i] = 1.0 / (1.0 + dtc + L.diag(ix, iy));
            x[i] = (mode == 1 || n0 == 0) ? u0[i] : U[(s * n + i) * N + n0 - 1];
        }
        bool failed = false;
        const int nint = mode == 0 ? 1 : N;
        for (int ni = 0; ni < nint; ++ni) {
            for (int j = 0; j < J; ++j) {
                __syncthreads();  // x complete
                // r = b - M x = dtf - L x, rh = r
                double v2[2] = {0.0, 0.0};  // ||b||^2, ||r||^2
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double ri = dtf - L.apply(x, i, ix, iy, dtc);
                    const double bi = x[i] + dtf;
                    r[i] = ri;
                    rh[i] = ri;
                    p[i] = 0.0;
                    v[i] = 0.0;
                    v2[0] = fma(bi, bi, v2[0]);
                    v2[1] = fma(ri, ri, v2[1]);
                }
                block_sum<2>(v2, red, ph);
                const double lim = rtol2 * v2[0];
                if (!(v2[1] > lim)) continue;  // x already solves the step
                double rho = 1.0, al = 1.0, om = 1.0, rho_new = v2[1];
                int it = 0;
                for (;;) {
                    const double beta = (rho_new / rho) * (al / om);
                    // p = r + beta (p - om v), y = D^{-1} p
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const double pi = fma(beta, fma(-om, v[i], p[i]), r[i]);
                        p[i] = pi;
                        y[i] = dinv[i] * pi;
                    }
                    __syncthreads();
                    // v = M y, (rh, v)
                    double w1[1] = {0.0};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const int iy = i / nx, ix = i - iy * nx;
                        const double vi = y[i] + L.apply(y, i, ix, iy, dtc);
                        v[i] = vi;
                        w1[0] = fma(rh[i], vi, w1[0]);
                    }
                    block_sum<1>(w1, red, ph);
                    if (!(w1[0] != 0.0)) {
                        failed = true;
                        break;
                    }
                    al = rho_new / w1[0];
                    // x += al y, s = r - al v (in r), z = D^{-1} s (in y), ||s||^2
                    double s1[1] = {0.0};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        x[i] = fma(al, y[i], x[i]);
                        const double si = fma(-al, v[i], r[i]);
                        r[i] = si;
                        y[i] = dinv[i] * si;
                        s1[0] = fma(si, si, s1[0]);
                    }
                    block_sum<1>(s1, red, ph);
                    ++it;
                    if (!(s1[0] > lim)) break;
                    // t = M z, (t, s), (t, t)
                    double w2[2] = {0.0, 0.0};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const int iy = i / nx, ix = i - iy * nx;
                        const double ti = y[i] + L.apply(y, i, ix, iy, dtc);
                        t[i] = ti;
                        w2[0] = fma(ti, r[i], w2[0]);
                        w2[1] = fma(ti, ti, w2[1]);
                    }
                    block_sum<2>(w2, red, ph);
                    if (!(w2[1] > 0.0)) {
                        failed = true;
                        break;
                    }
                    om = w2[0] / w2[1];
                    // x += om z, r = s - om t, ||r||^2, (rh, r)
                    double u2[2] = {0.0, 0.0};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        x[i] = fma(om, y[i], x[i]);
                        const double ri = fma(-om, t[i], r[i]);
                        r[i] = ri;
                        u2[0] = fma(ri, ri, u2[0]);
                        u2[1] = fma(rh[i], ri, u2[1]);
                    }
                    block_sum<2>(u2, red, ph);
                    if (!(u2[0] > lim)) break;
                    if (it >= maxit || !(om != 0.0) || !(u2[1] != 0.0)) {
                        failed = true;
                        break;
                    }
                    rho = rho_new;
                    rho_new = u2[1];
                }
                its_total += it;
            }
            if (mode == 1) {
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) out[(s * n + i) * N + ni] = x[i];
            }
        }
        if (mode == 0) {
            __syncthreads();  // x complete
            const double dTc = J * dtc;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int iy = i / nx, ix = i - iy * nx;
                const double Fi = x[i];
                const double LF = J * (L.apply(x, i, ix, iy, dtc) - dtc * Fi) + dTc * Fi;
                const double prev = n0 == 0 ? alpha * U[(s * n + i) * N + N - 1]
                                            : U[(s * n + i) * N + n0 - 1];
                out[(s * n + i) * N + n0] = (Fi + LF) - prev;
            }
        }
        if (failed && threadIdx.x == 0) ifail[s] = 1;
    }
    if (threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) b
__device__ __forceinline__ double2 cdotc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// c + a b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// ------------------------------------------------------------------- CGC (b), advection
// (lambda_k I + L_dT) q_k = p_k by Jacobi-preconditioned complex BiCGStab
// from zero (Hermitian inner products), in place in pio; adv = dT b0.
// Working storage: weights, dinv, x, r (also s), rh, p, v, y (also z), t.
__global__ void __launch_bounds__(kThreads2d) k_cgc_solve2d_bicgs(
    int64_t S, int K, int nx, double dTc, double adv, const double2* __restrict__ lam,
    const double* __restrict__ wdT, double rtol2, int maxit, double2* __restrict__ pio,
    const int* __restrict__ active, int* __restrict__ ifail,
    unsigned long long* __restrict__ itcount, double* __restrict__ gscr, int64_t per_cta) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red[2 * 3 * 32];
    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    double* W = gscr ? gscr + blockIdx.x * per_cta : dsm;
    double2* dinv = reinterpret_cast<double2*>(W + nf + (nf & 1));
    double2* x = dinv + n;
    double2* r = x + n;
    double2* rh = r + n;
    double2* p = rh + n;
    double2* v = p + n;
    double2* y = v + n;
    double2* t = y + n;
    const StencilAdv L{{W, W + nx * (nx + 1), nx}, adv};
    const double2 zero = make_double2(0.0, 0.0);
    int ph = 0;
    unsigned long long its_total = 0;
    for (int64_t item = blockIdx.x; item < S * K; item += gridDim.x) {
        const int64_t s = item / K;
        const int k = (int)(item - s * K);
        if (!active[s]) continue;
        __syncthreads();
        cpy_weights(W, wdT + s * nf, nf);
        __syncthreads();
        const double2 lk = lam[k];
        double b2[1] = {0.0};  // ||b||^2 (= ||r||^2 = (rh, r) at x = 0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int iy = i / nx, ix = i - iy * nx;
            dinv[i] = cdiv(make_double2(1.0, 0.0),
                           make_double2(lk.x + dTc + L.diag(ix, iy), lk.y));
            const double2 b = pio[(s * n + i) * K + k];
            x[i] = zero;
            r[i] = b;
            rh[i] = b;
            p[i] = zero;
            v[i] = zero;
            b2[0] = fma(b.x, b.x, fma(b.y, b.y, b2[0]));
        }
        block_sum<1>(b2, red, ph);
        const double lim = rtol2 * b2[0];
        bool failed = false;
        int it = 0;
        if (b2[0] > 0.0) {
            double2 rho = make_double2(1.0, 0.0), al = rho, om = rho;
            double2 rho_new = make_double2(b2[0], 0.0);
            for (;;) {
                const double2 beta = cmul(cdiv(rho_new, rho), cdiv(al, om));
                const double2 mom = make_double2(-om.x, -om.y);
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const double2 pi = cfma(beta, cfma(mom, v[i], p[i]), r[i]);
                    p[i] = pi;
                    y[i] = cmul(dinv[i], pi);
                }
                __syncthreads();
                double w1[2] = {0.0, 0.0};   // (rh, v)
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double2 yi = y[i];
                    const double2 ly = L.apply2(y, i, ix, iy, dTc);
                    const double2 vi = make_double2(lk.x * yi.x - lk.y * yi.y + ly.x,
                                                    lk.x * yi.y + lk.y * yi.x + ly.y);
                    v[i] = vi;
                    const double2 d = cdotc(rh[i], vi);
                    w1[0] += d.x;
                    w1[1] += d.y;
                }
                block_sum<2>(w1, red, ph);
                if (!(w1[0] != 0.0 || w1[1] != 0.0)) {
                    failed = true;
                    break;
                }
                al = cdiv(rho_new, make_double2(w1[0], w1[1]));
                const double2 mal = make_double2(-al.x, -al.y);
                double s1[1] = {0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    x[i] = cfma(al, y[i], x[i]);
                    const double2 si = cfma(mal, v[i], r[i]);
                    r[i] = si;
                    y[i] = cmul(dinv[i], si);
                    s1[0] = fma(si.x, si.x, fma(si.y, si.y, s1[0]));
                }
                block_sum<1>(s1, red, ph);
                ++it;
                if (!(s1[0] > lim)) break;
                double w3[3] = {0.0, 0.0, 0.0};   // (t, s), (t, t)
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double2 zi = y[i];
                    const double2 lz = L.apply2(y, i, ix, iy, dTc);
                    const double2 ti = make_double2(lk.x * zi.x - lk.y * zi.y + lz.x,
                                                    lk.x * zi.y + lk.y * zi.x + lz.y);
                    t[i] = ti;
                    const double2 d = cdotc(ti, r[i]);
                    w3[0] += d.x;
                    w3[1] += d.y;
                    w3[2] = fma(ti.x, ti.x, fma(ti.y, ti.y, w3[2]));
                }
                block_sum<3>(w3, red, ph);
                if (!(w3[2] > 0.0)) {
                    failed = true;
                    break;
                }
                om = make_double2(w3[0] / w3[2], w3[1] / w3[2]);
                const double2 mom2 = make_double2(-om.x, -om.y);
                double u3[3] = {0.0, 0.0, 0.0};   // ||r||^2, (rh, r)
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    x[i] = cfma(om, y[i], x[i]);
                    const double2 ri = cfma(mom2, t[i], r[i]);
                    r[i] = ri;
                    u3[0] = fma(ri.x, ri.x, fma(ri.y, ri.y, u3[0]));
                    const double2 d = cdotc(rh[i], ri);
                    u3[1] += d.x;
                    u3[2] += d.y;
                }
                block_sum<3>(u3, red, ph);
                if (!(u3[0] > lim)) break;
                if (it >= maxit || !(om.x != 0.0 || om.y != 0.0) || !(u3[1] != 0.0 || u3[2] != 0.0)) {
                    failed = true;
                    break;
                }
                rho = rho_new;
                rho_new = make_double2(u3[1], u3[2]);
            }
        }
        its_total += it;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) pio[(s * n + i) * K + k] = x[i];
        if (failed && threadIdx.x == 0) ifail[s] = 1;
    }
    if (threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
}

// ------------------------------------------------------------------- F, mixed
// The same propagator with every backward-Euler step solved by FP64
// iterative refinement around an FP32 Jacobi-PCG: the residual r = b - M x is
// formed once in FP64 and then updated in FP64 (r -= M d for each FP32
// correction d, x += d), so the solution is FP64-accurate (the stopping test
// is the same ||r||_2 <= rtol ||b||_2 on the FP64 residual) while the Krylov
// iterations run on the FP32 pipes.  Each inner solve stops at
// ||r32|| <= tin ||r32_0|| (or maxit); at most kMaxRef refinements per step.
// Working storage: x, r in FP64; FP32 weights, diagonal and the inner
// vectors d, r, z, p, q.  The FP64 weights are read from wdt (global).
constexpr int kMaxRef = 12;

struct Stencil32 {
    const float* wx;
    const float* wy;
    int nx;
    __device__ __forceinline__ float apply(const float* v, int i, int ix, int iy, float c) const {
        const float vi = v[i];
        const float* wr = wx + iy * (nx + 1) + ix;
        const float vw = ix > 0 ? v[i - 1] : 0.f;
        const float ve = ix < nx - 1 ? v[i + 1] : 0.f;
        const float vs = iy > 0 ? v[i - nx] : 0.f;
        const float vn = iy < nx - 1 ? v[i + nx] : 0.f;
        float acc = c * vi;
        acc = fmaf(wr[0], vi - vw, acc);
        acc = fmaf(wr[1], vi - ve, acc);
        acc = fmaf(wy[iy * nx + ix], vi - vs, acc);
        acc = fmaf(wy[(iy + 1) * nx + ix], vi - vn, acc);
        return acc;
    }
    __device__ __forceinline__ float wsum(int ix, int iy) const {
        const float* wr = wx + iy * (nx + 1) + ix;
        return wr[0] + wr[1] + wy[iy * nx + ix] + wy[(iy + 1) * nx + ix];
    }
};

// (I + L64) applied to the FP32 vector d, in FP64.
__device__ __forceinline__ double apply_m64(const Stencil& L, const float* d, int i, int ix,
                                            int iy, int nx, double c) {
    const double di = d[i];
    const double* wr = L.wx + iy * (nx + 1) + ix;
    const double dw = ix > 0 ? (double)d[i - 1] : 0.0;
    const double de = ix < nx - 1 ? (double)d[i + 1] : 0.0;
    const double ds = iy > 0 ? (double)d[i - nx] : 0.0;
    const double dn = iy < nx - 1 ? (double)d[i + nx] : 0.0;
    double acc = fma(c, di, di);
    acc = fma(wr[0], di - dw, acc);
    acc = fma(wr[1], di - de, acc);
    acc = fma(L.wy[iy * nx + ix], di - ds, acc);
    acc = fma(L.wy[(iy + 1) * nx + ix], di - dn, acc);
    return acc;
}

__global__ void __launch_bounds__(kThreads2d) k_fine2d_mixed(
    int64_t S, int N, int nx, int J, double dtc, double dtf, double alpha, int mode,
    const double* __restrict__ U, const double* __restrict__ u0, const double* __restrict__ wdt,
    double rtol2, float tin2, int maxit, double* __restrict__ out, const int* __restrict__ active,
    int* __restrict__ ifail, unsigned long long* __restrict__ itcount, double* __restrict__ gscr,
    int64_t per_cta) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red[2 * 3 * 32];
    __shared__ float red32[2 * 3 * 32];
    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    double* x = gscr ? gscr + blockIdx.x * per_cta : dsm;
    double* r = x + n;
    float* W32 = reinterpret_cast<float*>(r + n);
    float* dinv = W32 + nf;
    float* dv = dinv + n;
    float* rv = dv + n;
    float* zv = rv + n;
    float* pv = zv + n;
    float* qv = pv + n;
    const Stencil32 L32{W32, W32 + nx * (nx + 1), nx};
    const float c32 = (float)dtc;
    const int64_t items = mode == 0 ? S * N : S;
    int ph = 0, ph32 = 0;
    unsigned long long its_total = 0;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t s = mode == 0 ? item / N : item;
        const int n0 = mode == 0 ? (int)(item - s * N) : 0;
        if (!active[s]) continue;
        const double* wg = wdt + s * nf;
        const Stencil L{wg, wg + nx * (nx + 1), nx};
        __syncthreads();  // the previous item's epilogue has read its vectors
        for (int e = threadIdx.x; e < nf; e += blockDim.x) W32[e] = (float)wg[e];
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int iy = i / nx, ix = i - iy * nx;
            dinv[i] = 1.f / (1.f + c32 + L32.wsum(ix, iy));
            x[i] = (mode == 1 || n0 == 0) ? u0[i] : U[(s * n + i) * N + n0 - 1];
        }
        bool failed = false;
        const int nint = mode == 0 ? 1 : N;
        for (int ni = 0; ni < nint; ++ni) {
            for (int j = 0; j < J; ++j) {
                __syncthreads();  // x complete
                // FP64 residual of the step at x = x_old: r = dtf - L x
                double v2[2] = {0.0, 0.0};  // ||b||^2, ||r||^2
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double ri = dtf - L.apply(x, i, ix, iy, dtc);
                    const double bi = x[i] + dtf;
                    r[i] = ri;
                    v2[0] = fma(bi, bi, v2[0]);
                    v2[1] = fma(ri, ri, v2[1]);
                }
                block_sum<2>(v2, red, ph);
                const double lim = rtol2 * v2[0];
                double rr64 = v2[1];
                int ref = 0;
                while (rr64 > lim) {
                    if (ref++ >= kMaxRef) {
                        failed = true;
                        break;
                    }
                    // inner FP32 PCG: (I + L32) d = r / sigma, d0 = 0, sigma the RMS of
                    // r (keeps the FP32 values and their squares far from underflow)
                    const double sigma = sqrt(rr64 / n), isig = 1.0 / sigma;
                    float v3[3] = {0.f, 0.f, 0.f};  // r.z, ||r||^2
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const float ri = (float)(r[i] * isig);
                        const float zi = dinv[i] * ri;
                        dv[i] = 0.f;
                        rv[i] = ri;
                        zv[i] = zi;
                        pv[i] = zi;
                        v3[0] = fmaf(ri, zi, v3[0]);
                        v3[1] = fmaf(ri, ri, v3[1]);
                    }
                    float w2[2] = {v3[0], v3[1]};
                    block_sum32<2>(w2, red32, ph32);
                    float rz = w2[0];
                    const float ilim = tin2 * w2[1];
                    float w1[1] = {0.f};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const int iy = i / nx, ix = i - iy * nx;
                        const float qi = pv[i] + L32.apply(pv, i, ix, iy, c32);
                        qv[i] = qi;
                        w1[0] = fmaf(pv[i], qi, w1[0]);
                    }
                    block_sum32<1>(w1, red32, ph32);
                    float pq = w1[0];
                    int it = 0;
                    for (;;) {
                        const float a = rz / pq;
                        float u2[2] = {0.f, 0.f};
                        for (int i = threadIdx.x; i < n; i += blockDim.x) {
                            dv[i] = fmaf(a, pv[i], dv[i]);
                            const float ri = fmaf(-a, qv[i], rv[i]);
                            const float zi = dinv[i] * ri;
                            rv[i] = ri;
                            zv[i] = zi;
                            u2[0] = fmaf(ri, ri, u2[0]);
                            u2[1] = fmaf(ri, zi, u2[1]);
                        }
                        block_sum32<2>(u2, red32, ph32);
                        ++it;
                        if (!(u2[0] > ilim) || it >= maxit) break;
                        const float rzn = u2[1];
                        const float beta = rzn / rz;
                        rz = rzn;
                        float y1[1] = {0.f};
                        for (int i = threadIdx.x; i < n; i += blockDim.x) {
                            const int iy = i / nx, ix = i - iy * nx;
                            const float zi = zv[i];
                            const float pi = fmaf(beta, pv[i], zi);
                            const float qi = fmaf(beta, qv[i], zi + L32.apply(zv, i, ix, iy, c32));
                            pv[i] = pi;
                            qv[i] = qi;
                            y1[0] = fmaf(pi, qi, y1[0]);
                        }
                        block_sum32<1>(y1, red32, ph32);
                        pq = y1[0];
                    }
                    its_total += it;
                    // FP64 update: x += sigma d, r -= sigma (I + L) d   (d complete
                    // after the last reduction)
                    double z1[1] = {0.0};
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        const int iy = i / nx, ix = i - iy * nx;
                        x[i] = fma(sigma, (double)dv[i], x[i]);
                        const double ri = fma(-sigma, apply_m64(L, dv, i, ix, iy, nx, dtc), r[i]);
                        r[i] = ri;
                        z1[0] = fma(ri, ri, z1[0]);
                    }
                    block_sum<1>(z1, red, ph);
                    rr64 = z1[0];
                }
            }
            if (mode == 1) {
                __syncthreads();
                for (int i = threadIdx.x; i < n; i += blockDim.x) out[(s * n + i) * N + ni] = x[i];
            }
        }
        if (mode == 0) {
            __syncthreads();  // x complete
            const double dTc = J * dtc;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int iy = i / nx, ix = i - iy * nx;
                const double Fi = x[i];
                const double LF = J * (L.apply(x, i, ix, iy, dtc) - dtc * Fi) + dTc * Fi;
                const double prev = n0 == 0 ? alpha * U[(s * n + i) * N + N - 1]
                                            : U[(s * n + i) * N + n0 - 1];
                out[(s * n + i) * N + n0] = (Fi + LF) - prev;
            }
        }
        if (failed && threadIdx.x == 0) ifail[s] = 1;
    }
    if (threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
}

// ------------------------------------------------------------------- CGC (b)
// item (s, k), k = 0..K-1: solves (lambda_k I + L_dT) q = p in place in
// p[s][i][k] (layout [S][n_unknowns][K]).
__global__ void __launch_bounds__(kThreads2d) k_cgc_solve2d(
    int64_t S, int K, int nx, double dTc, const double2* __restrict__ lam,
    const double* __restrict__ wdT, double rtol2, int maxit, double2* __restrict__ pio,
    const int* __restrict__ active, int* __restrict__ ifail,
    unsigned long long* __restrict__ itcount, double* __restrict__ gscr, int64_t per_cta) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red[2 * 3 * 32];
    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    double* W = gscr ? gscr + blockIdx.x * per_cta : dsm;
    double2* dinv = reinterpret_cast<double2*>(W + nf + (nf & 1));
    double2* x = dinv + n;
    double2* r = x + n;
    double2* z = r + n;
    double2* p = z + n;
    double2* q = p + n;
    const Stencil L{W, W + nx * (nx + 1), nx};
    int ph = 0;
    unsigned long long its_total = 0;
    for (int64_t item = blockIdx.x; item < S * K; item += gridDim.x) {
        const int64_t s = item / K;
        const int k = (int)(item - s * K);
        if (!active[s]) continue;
        __syncthreads();
        cpy_weights(W, wdT + s * nf, nf);
        __syncthreads();
        const double2 lk = lam[k];
        double v3[3] = {0.0, 0.0, 0.0};  // ||b||^2, r.z (complex)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int iy = i / nx, ix = i - iy * nx;
            const double dr = lk.x + dTc + L.wsum(ix, iy), di = lk.y;
            const double den = dr * dr + di * di;
            const double2 dv = make_double2(dr / den, -di / den);
            dinv[i] = dv;
            const double2 b = pio[(s * n + i) * K + k];
            const double2 zi = make_double2(dv.x * b.x - dv.y * b.y, dv.x * b.y + dv.y * b.x);
            x[i] = make_double2(0.0, 0.0);
            r[i] = b;
            z[i] = zi;
            p[i] = zi;
            v3[0] = fma(b.x, b.x, fma(b.y, b.y, v3[0]));
            v3[1] = fma(b.x, zi.x, fma(-b.y, zi.y, v3[1]));
            v3[2] = fma(b.x, zi.y, fma(b.y, zi.x, v3[2]));
        }
        block_sum<3>(v3, red, ph);
        const double lim = rtol2 * v3[0];
        bool failed = false;
        int it = 0;
        if (v3[0] > 0.0) {
            double rzr = v3[1], rzi = v3[2];
            // q = M p, p.q
            double v2[2] = {0.0, 0.0};
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int iy = i / nx, ix = i - iy * nx;
                const double2 pi = p[i];
                const double2 lp = L.apply2(p, i, ix, iy, dTc);
                const double2 qi = make_double2(lk.x * pi.x - lk.y * pi.y + lp.x,
                                                lk.x * pi.y + lk.y * pi.x + lp.y);
                q[i] = qi;
                v2[0] = fma(pi.x, qi.x, fma(-pi.y, qi.y, v2[0]));
                v2[1] = fma(pi.x, qi.y, fma(pi.y, qi.x, v2[1]));
            }
            block_sum<2>(v2, red, ph);
            double pqr = v2[0], pqi = v2[1];
            for (;;) {
                // a = rz / pq
                const double den = pqr * pqr + pqi * pqi;
                const double ar = (rzr * pqr + rzi * pqi) / den, ai = (rzi * pqr - rzr * pqi) / den;
                double u3[3] = {0.0, 0.0, 0.0};  // ||r||^2, r.z
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const double2 pi = p[i], qi = q[i], dv = dinv[i];
                    double2 xi = x[i], ri = r[i];
                    xi.x = fma(ar, pi.x, fma(-ai, pi.y, xi.x));
                    xi.y = fma(ar, pi.y, fma(ai, pi.x, xi.y));
                    ri.x = fma(-ar, qi.x, fma(ai, qi.y, ri.x));
                    ri.y = fma(-ar, qi.y, fma(-ai, qi.x, ri.y));
                    const double2 zi = make_double2(dv.x * ri.x - dv.y * ri.y, dv.x * ri.y + dv.y * ri.x);
                    x[i] = xi;
                    r[i] = ri;
                    z[i] = zi;
                    u3[0] = fma(ri.x, ri.x, fma(ri.y, ri.y, u3[0]));
                    u3[1] = fma(ri.x, zi.x, fma(-ri.y, zi.y, u3[1]));
                    u3[2] = fma(ri.x, zi.y, fma(ri.y, zi.x, u3[2]));
                }
                block_sum<3>(u3, red, ph);
                ++it;
                if (!(u3[0] > lim)) break;
                if (it >= maxit) {
                    failed = true;
                    break;
                }
                // beta = rz_new / rz
                const double dd = rzr * rzr + rzi * rzi;
                const double br = (u3[1] * rzr + u3[2] * rzi) / dd, bi = (u3[2] * rzr - u3[1] * rzi) / dd;
                rzr = u3[1];
                rzi = u3[2];
                double w2[2] = {0.0, 0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const double2 zi = z[i], po = p[i], qo = q[i];
                    const double2 lz = L.apply2(z, i, ix, iy, dTc);
                    const double2 mz = make_double2(lk.x * zi.x - lk.y * zi.y + lz.x,
                                                    lk.x * zi.y + lk.y * zi.x + lz.y);
                    const double2 pn = make_double2(fma(br, po.x, fma(-bi, po.y, zi.x)),
                                                    fma(br, po.y, fma(bi, po.x, zi.y)));
                    const double2 qn = make_double2(fma(br, qo.x, fma(-bi, qo.y, mz.x)),
                                                    fma(br, qo.y, fma(bi, qo.x, mz.y)));
                    p[i] = pn;
                    q[i] = qn;
                    w2[0] = fma(pn.x, qn.x, fma(-pn.y, qn.y, w2[0]));
                    w2[1] = fma(pn.x, qn.y, fma(pn.y, qn.x, w2[1]));
                }
                block_sum<2>(w2, red, ph);
                pqr = w2[0];
                pqi = w2[1];
            }
        }
        its_total += it;
        for (int i = threadIdx.x; i < n; i += blockDim.x) pio[(s * n + i) * K + k] = x[i];
        if (failed && threadIdx.x == 0) ifail[s] = 1;
    }
    if (threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
}

// ------------------------------------------------------------------- CGC (b), mixed
// The shifted solves by FP64 iterative refinement around an FP32 Jacobi-COCG,
// as for F: x accumulates in FP64 in the output p itself, the residual is
// kept and updated in FP64 (complex), each correction equation is scaled by
// the residual's RMS and solved in FP32 to tin; the stopping test is
// ||r||_2 <= rtol ||p_k||_2 on the FP64 residual.  Working storage: r in FP64
// (complex); FP32 weights, complex diagonal and the inner vectors d, r, z, p, q.
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// L32 applied to a complex FP32 vector (real weights).
__device__ __forceinline__ float2 apply2f(const Stencil32& L, const float2* v, int i, int ix,
                                         int iy, float c) {
    const int nx = L.nx;
    const float2 vi = v[i];
    const float2 z = make_float2(0.f, 0.f);
    const float* wr = L.wx + iy * (nx + 1) + ix;
    const float2 vw = ix > 0 ? v[i - 1] : z;
    const float2 ve = ix < nx - 1 ? v[i + 1] : z;
    const float2 vs = iy > 0 ? v[i - nx] : z;
    const float2 vn = iy < nx - 1 ? v[i + nx] : z;
    const float a0 = wr[0], a1 = wr[1], a2 = L.wy[iy * nx + ix], a3 = L.wy[(iy + 1) * nx + ix];
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

// (lambda I + L64) applied to the complex FP32 vector d, in FP64.
__device__ __forceinline__ double2 apply_shift64(const Stencil& L, const float2* d, int i, int ix,
                                                 int iy, int nx, double c, double2 lk) {
    const float2 df = d[i];
    const double dr = df.x, di = df.y;
    const double* wr = L.wx + iy * (nx + 1) + ix;
    const float2 z = make_float2(0.f, 0.f);
    const float2 fw = ix > 0 ? d[i - 1] : z;
    const float2 fe = ix < nx - 1 ? d[i + 1] : z;
    const float2 fs = iy > 0 ? d[i - nx] : z;
    const float2 fn = iy < nx - 1 ? d[i + nx] : z;
    const double a0 = wr[0], a1 = wr[1], a2 = L.wy[iy * nx + ix], a3 = L.wy[(iy + 1) * nx + ix];
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

__global__ void __launch_bounds__(kThreads2d) k_cgc_solve2d_mixed(
    int64_t S, int K, int nx, double dTc, const double2* __restrict__ lam,
    const double* __restrict__ wdT, double rtol2, float tin2, int maxit,
    double2* __restrict__ pio, const int* __restrict__ active, int* __restrict__ ifail,
    unsigned long long* __restrict__ itcount, double* __restrict__ gscr, int64_t per_cta) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ double red[2 * 3 * 32];
    __shared__ float red32[2 * 3 * 32];
    const int n = nx * nx, nf = 2 * nx * (nx + 1);
    double2* r = reinterpret_cast<double2*>(gscr ? gscr + blockIdx.x * per_cta : dsm);
    float* W32 = reinterpret_cast<float*>(r + n);
    float2* dinv = reinterpret_cast<float2*>(W32 + nf + (nf & 1));
    float2* dv = dinv + n;
    float2* rv = dv + n;
    float2* zv = rv + n;
    float2* pv = zv + n;
    float2* qv = pv + n;
    const Stencil32 L32{W32, W32 + nx * (nx + 1), nx};
    const float c32 = (float)dTc;
    int ph = 0, ph32 = 0;
    unsigned long long its_total = 0;
    for (int64_t item = blockIdx.x; item < S * K; item += gridDim.x) {
        const int64_t s = item / K;
        const int k = (int)(item - s * K);
        if (!active[s]) continue;
        const double* wg = wdT + s * nf;
        const Stencil L{wg, wg + nx * (nx + 1), nx};
        const double2 lk = lam[k];
        const float2 lk32 = make_float2((float)lk.x, (float)lk.y);
        __syncthreads();  // the previous item is done with the shared vectors
        for (int e = threadIdx.x; e < nf; e += blockDim.x) W32[e] = (float)wg[e];
        __syncthreads();
        double v1[1] = {0.0};  // ||b||^2
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const int iy = i / nx, ix = i - iy * nx;
            const float dr = lk32.x + c32 + L32.wsum(ix, iy), di = lk32.y;
            const float den = dr * dr + di * di;
            dinv[i] = make_float2(dr / den, -di / den);
            double2* o = pio + (s * n + i) * K + k;
            const double2 b = *o;
            r[i] = b;
            *o = make_double2(0.0, 0.0);   // x accumulates here
            v1[0] = fma(b.x, b.x, fma(b.y, b.y, v1[0]));
        }
        block_sum<1>(v1, red, ph);
        const double lim = rtol2 * v1[0];
        double rr64 = v1[0];
        bool failed = false;
        int ref = 0;
        while (rr64 > lim) {
            if (ref++ >= kMaxRef) {
                failed = true;
                break;
            }
            const double sigma = sqrt(rr64 / n), isig = 1.0 / sigma;
            // inner FP32 COCG: (lambda I + L32) d = r / sigma, d0 = 0
            float v3[3] = {0.f, 0.f, 0.f};  // ||r||^2, r.z (complex, unconjugated)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const double2 rd = r[i];
                const float2 ri = make_float2((float)(rd.x * isig), (float)(rd.y * isig));
                const float2 zi = cmulf(dinv[i], ri);
                dv[i] = make_float2(0.f, 0.f);
                rv[i] = ri;
                zv[i] = zi;
                pv[i] = zi;
                v3[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, v3[0]));
                v3[1] = fmaf(ri.x, zi.x, fmaf(-ri.y, zi.y, v3[1]));
                v3[2] = fmaf(ri.x, zi.y, fmaf(ri.y, zi.x, v3[2]));
            }
            block_sum32<3>(v3, red32, ph32);
            const float ilim = tin2 * v3[0];
            float rzr = v3[1], rzi = v3[2];
            // q = M p, p.q
            float w2[2] = {0.f, 0.f};
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int iy = i / nx, ix = i - iy * nx;
                const float2 pi = pv[i];
                const float2 lp = apply2f(L32, pv, i, ix, iy, c32);
                const float2 qi = make_float2(lk32.x * pi.x - lk32.y * pi.y + lp.x,
                                              lk32.x * pi.y + lk32.y * pi.x + lp.y);
                qv[i] = qi;
                w2[0] = fmaf(pi.x, qi.x, fmaf(-pi.y, qi.y, w2[0]));
                w2[1] = fmaf(pi.x, qi.y, fmaf(pi.y, qi.x, w2[1]));
            }
            block_sum32<2>(w2, red32, ph32);
            float pqr = w2[0], pqi = w2[1];
            int it = 0;
            for (;;) {
                const float den = pqr * pqr + pqi * pqi;
                const float ar = (rzr * pqr + rzi * pqi) / den, ai = (rzi * pqr - rzr * pqi) / den;
                float u3[3] = {0.f, 0.f, 0.f};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const float2 pi = pv[i], qi = qv[i], dvi = dinv[i];
                    float2 di = dv[i], ri = rv[i];
                    di.x = fmaf(ar, pi.x, fmaf(-ai, pi.y, di.x));
                    di.y = fmaf(ar, pi.y, fmaf(ai, pi.x, di.y));
                    ri.x = fmaf(-ar, qi.x, fmaf(ai, qi.y, ri.x));
                    ri.y = fmaf(-ar, qi.y, fmaf(-ai, qi.x, ri.y));
                    const float2 zi = cmulf(dvi, ri);
                    dv[i] = di;
                    rv[i] = ri;
                    zv[i] = zi;
                    u3[0] = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, u3[0]));
                    u3[1] = fmaf(ri.x, zi.x, fmaf(-ri.y, zi.y, u3[1]));
                    u3[2] = fmaf(ri.x, zi.y, fmaf(ri.y, zi.x, u3[2]));
                }
                block_sum32<3>(u3, red32, ph32);
                ++it;
                if (!(u3[0] > ilim) || it >= maxit) break;
                const float dd = rzr * rzr + rzi * rzi;
                const float br = (u3[1] * rzr + u3[2] * rzi) / dd, bi = (u3[2] * rzr - u3[1] * rzi) / dd;
                rzr = u3[1];
                rzi = u3[2];
                float y2[2] = {0.f, 0.f};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int iy = i / nx, ix = i - iy * nx;
                    const float2 zi = zv[i], po = pv[i], qo = qv[i];
                    const float2 lz = apply2f(L32, zv, i, ix, iy, c32);
                    const float2 mz = make_float2(lk32.x * zi.x - lk32.y * zi.y + lz.x,
                                                  lk32.x * zi.y + lk32.y * zi.x + lz.y);
                    const float2 pn = make_float2(fmaf(br, po.x, fmaf(-bi, po.y, zi.x)),
                                                  fmaf(br, po.y, fmaf(bi, po.x, zi.y)));
                    const float2 qn = make_float2(fmaf(br, qo.x, fmaf(-bi, qo.y, mz.x)),
                                                  fmaf(br, qo.y, fmaf(bi, qo.x, mz.y)));
                    pv[i] = pn;
                    qv[i] = qn;
                    y2[0] = fmaf(pn.x, qn.x, fmaf(-pn.y, qn.y, y2[0]));
                    y2[1] = fmaf(pn.x, qn.y, fmaf(pn.y, qn.x, y2[1]));
                }
                block_sum32<2>(y2, red32, ph32);
                pqr = y2[0];
                pqi = y2[1];
            }
            its_total += it;
            // FP64 update: x += sigma d (in the output), r -= sigma (lambda I + L) d
            double z1[1] = {0.0};
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int iy = i / nx, ix = i - iy * nx;
                double2* o = pio + (s * n + i) * K + k;
                const float2 di = dv[i];
                double2 xo = *o;
                xo.x = fma(sigma, (double)di.x, xo.x);
                xo.y = fma(sigma, (double)di.y, xo.y);
                *o = xo;
                const double2 md = apply_shift64(L, dv, i, ix, iy, nx, dTc, lk);
                double2 ri = r[i];
                ri.x = fma(-sigma, md.x, ri.x);
                ri.y = fma(-sigma, md.y, ri.y);
                r[i] = ri;
                z1[0] = fma(ri.x, ri.x, fma(ri.y, ri.y, z1[0]));
            }
            block_sum<1>(z1, red, ph);
            rr64 = z1[0];
        }
        if (failed && threadIdx.x == 0) ifail[s] = 1;
    }
    if (threadIdx.x == 0 && itcount && its_total) atomicAdd(itcount, its_total);
}

int num_sms() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

int max_dyn_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Doubles of working storage per system.
int64_t per_system(int kind, int nx) {
    const int64_t n = (int64_t)nx * nx, nf = 2 * (int64_t)nx * (nx + 1);
    if (kind == 2) return 2 * n + (nf + 6 * n + 1) / 2;   // FP64 x, r; FP32 rest
    if (kind == 3) return 2 * n + (nf + (nf & 1) + 12 * n + 1) / 2;  // FP64 r; FP32 rest
    if (kind == 4) return nf + 8 * n;                       // BiCGStab, real
    if (kind == 5) return nf + (nf & 1) + 16 * n;           // BiCGStab, complex
    return kind == 0 ? nf + 6 * n : nf + (nf & 1) + 12 * n;
}

}  // namespace

Plan2D plan_2d(int kind, int nx, int64_t items, bool force_cluster) {
    Plan2D pl;
    const int64_t per = per_system(kind, nx);
    const int64_t bytes = per * 8;
    const int sm = num_sms();
    const int static_bytes = 2 * 3 * 32 * 8;
    if ((kind == 2 || kind == 3) && (force_cluster || bytes + static_bytes > max_dyn_smem())) {
        // the mixed system on a thread-block cluster, if one holds it
        const ClusterPlan2D cp = kind == 2 ? fine2d_cluster_plan(nx) : cgc2d_cluster_plan(nx);
        if (cp.CL > 0) {
            pl.cl = cp;
            pl.grid = (int64_t)cp.CL * std::min<int64_t>(cp.clusters, std::max<int64_t>(items, 1));
            pl.scratch_doubles = cp.scratch_per_cta * pl.grid;
            return pl;
        }
    }
    if (bytes + static_bytes <= max_dyn_smem()) {
        pl.smem = (int)bytes;
        int occ = 0;
        if (kind == 0) {
            cudaFuncSetAttribute(k_fine2d, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fine2d, kThreads2d, pl.smem);
        } else if (kind == 2) {
            cudaFuncSetAttribute(k_fine2d_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pl.smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fine2d_mixed, kThreads2d,
                                                          pl.smem);
        } else if (kind == 4) {
            cudaFuncSetAttribute(k_fine2d_bicgs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pl.smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fine2d_bicgs, kThreads2d,
                                                          pl.smem);
        } else if (kind == 5) {
            cudaFuncSetAttribute(k_cgc_solve2d_bicgs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pl.smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgc_solve2d_bicgs, kThreads2d,
                                                          pl.smem);
        } else if (kind == 3) {
            cudaFuncSetAttribute(k_cgc_solve2d_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pl.smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgc_solve2d_mixed, kThreads2d,
                                                          pl.smem);
        } else {
            cudaFuncSetAttribute(k_cgc_solve2d, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.smem);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgc_solve2d, kThreads2d, pl.smem);
        }
        pl.grid = (int64_t)sm * (occ > 0 ? occ : 1);
        pl.per_cta = 0;
    } else {
        // working storage in global memory: two CTAs per SM, one slice each
        pl.smem = 0;
        pl.grid = 2 * (int64_t)sm;
        pl.per_cta = per + (per & 1);
    }
    if (pl.grid > items) pl.grid = items;
    if (pl.grid < 1) pl.grid = 1;
    pl.scratch_doubles = pl.per_cta * pl.grid;
    return pl;
}

void launch_fine2d(const Plan2D& pl, int64_t S, int N, int nx, int J, double dtc, double dtf,
                   double adv, double alpha, int mode, const double* U, const double* u0,
                   const double* wdt, double rtol, int maxit, double* out, const int* active,
                   int* ifail, unsigned long long* itcount, double* scratch, cudaStream_t st) {
    if (S == 0) return;
    if (adv != 0.0)
        k_fine2d_bicgs<<<(unsigned)pl.grid, kThreads2d, pl.smem, st>>>(
            S, N, nx, J, dtc, dtf, adv, alpha, mode, U, u0, wdt, rtol * rtol, maxit, out, active,
            ifail, itcount, pl.per_cta ? scratch : nullptr, pl.per_cta);
    else
        k_fine2d<<<(unsigned)pl.grid, kThreads2d, pl.smem, st>>>(
            S, N, nx, J, dtc, dtf, alpha, mode, U, u0, wdt, rtol * rtol, maxit, out, active,
            ifail, itcount, pl.per_cta ? scratch : nullptr, pl.per_cta);
}

void launch_fine2d_mixed(const Plan2D& pl, int64_t S, int N, int nx, int J, double dtc,
                         double dtf, double alpha, int mode, const double* U, const double* u0,
                         const double* wdt, double rtol, double tin, int maxit, double* out,
                         const int* active, int* ifail, unsigned long long* itcount,
                         double* scratch, cudaStream_t st) {
    if (S == 0) return;
    if (pl.cl.CL > 0) {
        launch_fine2d_mixed_cl(pl.cl, S, N, nx, J, dtc, dtf, alpha, mode, U, u0, wdt, rtol, tin,
                               maxit, out, active, ifail, itcount, st);
        return;
    }
    k_fine2d_mixed<<<(unsigned)pl.grid, kThreads2d, pl.smem, st>>>(
        S, N, nx, J, dtc, dtf, alpha, mode, U, u0, wdt, rtol * rtol, (float)(tin * tin), maxit,
        out, active, ifail, itcount, pl.per_cta ? scratch : nullptr, pl.per_cta);
}

void launch_cgc_solve2d_mixed(const Plan2D& pl, int64_t S, int K, int nx, double dTc,
                              const double2* lam, const double* wdT, double rtol, double tin,
                              int maxit, Cplx<double>* p, const int* active, int* ifail,
                              unsigned long long* itcount, double* scratch, cudaStream_t st) {
    if (S == 0) return;
    if (pl.cl.CL > 0) {
        launch_cgc_solve2d_mixed_cl(pl.cl, S, K, nx, dTc, lam, wdT, rtol, tin, maxit, p, active,
                                    ifail, itcount, scratch, pl.grid, st);
        return;
    }
    k_cgc_solve2d_mixed<<<(unsigned)pl.grid, kThreads2d, pl.smem, st>>>(
        S, K, nx, dTc, lam, wdT, rtol * rtol, (float)(tin * tin), maxit,
        reinterpret_cast<double2*>(p), active, ifail, itcount, pl.per_cta ? scratch : nullptr,
        pl.per_cta);
}

void launch_cgc_solve2d(const Plan2D& pl, int64_t S, int K, int nx, double dTc, double adv,
                        const double2* lam, const double* wdT, double rtol, int maxit,
                        Cplx<double>* p, const int* active, int* ifail,
                        unsigned long long* itcount, double* scratch, cudaStream_t st) {
    if (S == 0) return;
    if (adv != 0.0)
        k_cgc_solve2d_bicgs<<<(unsigned)pl.grid, kThreads2d, pl.smem, st>>>(
            S, K, nx, dTc, adv, lam, wdT, rtol * rtol, maxit, reinterpret_cast<double2*>(p),
            active, ifail, itcount, pl.per_cta ? scratch : nullptr, pl.per_cta);
    else
        k_cgc_solve2d<<<(unsigned)pl.grid, kThreads2d, pl.smem, st>>>(
            S, K, nx, dTc, lam, wdT, rtol * rtol, maxit, reinterpret_cast<double2*>(p), active,
            ifail, itcount, pl.per_cta ? scratch : nullptr, pl.per_cta);
}

}  // namespace klecgc
