// Banded direct solves for small 2D grids (nx <= kBandMaxNx): the fine
// propagator's backward-Euler systems (I + dt(A + cI) + convection) and the
// CGC's shifted systems (lambda_k I + dT(A + cI) + convection), eq. three
// steps (b).  In the natural ordering i = iy*nx + ix the five-point operator
// has bandwidth nx, and LU without pivoting keeps the band (the matrices are
// diagonally dominant M-matrices, also with the upwind convection; the
// complex shift adds a positive real part), so each matrix is factored once
// per solve and every step or shifted solve is one forward and one backward
// substitution of bandwidth nx.
//
// Band storage: row i holds columns i - nx .. i + nx at offsets 0 .. 2 nx
// (W = 2 nx + 1 values); after factoring, the strictly lower part holds the
// multipliers of the unit lower factor, the upper part U, and the diagonal
// 1 / U_ii.
//
// Factoring: one warp per matrix; for each pivot k the lanes form the nx
// multipliers of rows k+1 .. k+nx, then update the nx x nx trailing block.
// Substitution: one thread per right-hand side, vectors in the library's
// [S][n][N] (or [S][n][K]) layout, so a warp of consecutive intervals (or
// frequencies) of one sample reads each row of the shared factors once
// (broadcast) and its vector entries coalesced.
#include "common.cuh"

namespace klecgc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct CxOps;
template <>
struct CxOps<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double fms(double acc, double a, double b) { return fma(-a, b, acc); }
    static __device__ __forceinline__ double inv(double a) { return 1.0 / a; }
    static __device__ __forceinline__ double make(double re, double) { return re; }
    static __device__ __forceinline__ double add_re(double a, double r) { return a + r; }
};
template <>
struct CxOps<double2> {
    static __device__ __forceinline__ double2 mul(double2 a, double2 b) {
        return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    }
    static __device__ __forceinline__ double2 fms(double2 acc, double2 a, double2 b) {
        return make_double2(fma(-a.x, b.x, fma(a.y, b.y, acc.x)), fma(-a.x, b.y, fma(-a.y, b.x, acc.y)));
    }
    static __device__ __forceinline__ double2 inv(double2 a) {
        const double d = a.x * a.x + a.y * a.y;
        return make_double2(a.x / d, -a.y / d);
    }
    static __device__ __forceinline__ double2 make(double re, double im) { return make_double2(re, im); }
    static __device__ __forceinline__ double2 add_re(double2 a, double r) { return make_double2(a.x + r, a.y); }
};

// Face weights of cell (ix, iy): x-faces [nx][nx+1], then y-faces [nx+1][nx].
struct Faces {
    double wW, wE, wS, wN;
};
__device__ __forceinline__ Faces faces(const double* w, int nx, int ix, int iy) {
    const double* wx = w + iy * (nx + 1) + ix;
    const double* wy = w + nx * (nx + 1);
    return {wx[0], wx[1], wy[iy * nx + ix], wy[(iy + 1) * nx + ix]};
}

// Builds scale * (A + cI) + convection + shift I in band form for matrix m
// (sample s = m / per_sample) and factors it.  w: scale-weighted faces
// (scale a / h^2); cs = scale c; adv = scale b0; shift per matrix from
// shifts[m % per_sample] (complex) or 1 (real, shifts == nullptr).
template <typename T>
__global__ void __launch_bounds__(128) k_band_factor(int64_t nmat, int per_sample, int nx,
                                                     const double* __restrict__ w, double cs,
                                                     double adv,
                                                     const double2* __restrict__ shifts,
                                                     T* __restrict__ B) {
    using O = CxOps<T>;
    const int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (m >= nmat) return;   // whole warps
    const int64_t s = m / per_sample;
    const int n = nx * nx, bw = nx, W = 2 * nx + 1;
    T* Bm = B + m * (int64_t)n * W;
    const double* ws = w + s * (int64_t)(2 * nx * (nx + 1));
    const double2 sh = shifts ? shifts[m % per_sample] : make_double2(1.0, 0.0);
    for (int i = lane; i < n; i += 32) {
        const int iy = i / nx, ix = i - iy * nx;
        const Faces f = faces(ws, nx, ix, iy);
        T* row = Bm + (int64_t)i * W;
        for (int o = 0; o < W; ++o) row[o] = O::make(0.0, 0.0);
        const double c1 = adv * (iy + 1), c2 = adv * (ix + 1);   // upwind: u_W, u_S
        row[bw] = O::make(sh.x + cs + f.wW + f.wE + f.wS + f.wN + c1 + c2, sh.y);
        if (ix > 0) row[bw - 1] = O::make(-f.wW - c1, 0.0);
        if (ix < nx - 1) row[bw + 1] = O::make(-f.wE, 0.0);
        if (iy > 0) row[0] = O::make(-f.wS - c2, 0.0);
        if (iy < nx - 1) row[2 * bw] = O::make(-f.wN, 0.0);
    }
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        T* rk = Bm + (int64_t)k * W;
        const T pinv = O::inv(rk[bw]);
        const int rmax = min(bw, n - 1 - k);   // rows / columns after k in the band
        // multipliers l_ik = B_ik / U_kk, i = k+1 .. k+rmax (offset k - i + bw)
        for (int r = 1 + lane; r <= rmax; r += 32) {
            T* bik = Bm + (int64_t)(k + r) * W + (bw - r);
            *bik = O::mul(*bik, pinv);
        }
        __syncwarp();
        // trailing update B_ij -= l_ik U_kj, i, j = k+1 .. k+rmax
        for (int e = lane; e < rmax * rmax; e += 32) {
            const int r = 1 + e / rmax, c = 1 + e - (r - 1) * rmax;
            const int i = k + r, j = k + c;
            T* rowi = Bm + (int64_t)i * W;
            const T lik = rowi[k - i + bw];
            T& bij = rowi[j - i + bw];
            bij = O::fms(bij, lik, rk[j - k + bw]);
        }
        __syncwarp();
        if (lane == 0) rk[bw] = pinv;
        __syncwarp();
    }
}

// x <- M^{-1} x for one right-hand side with factors Bm, vector entries at
// x[i * stride] (i = 0 .. n-1).
template <typename T>
__device__ __forceinline__ void band_solve(const T* __restrict__ Bm, int nx, T* x, int64_t stride) {
    using O = CxOps<T>;
    const int n = nx * nx, bw = nx, W = 2 * nx + 1;
    // forward: y_i = x_i - sum_k l_ik y_k (unit lower factor)
    for (int i = 1; i < n; ++i) {
        const T* row = Bm + (int64_t)i * W;
        const int k0 = max(0, i - bw);
        T a0 = x[(int64_t)i * stride], a1 = O::make(0.0, 0.0);
        int k = k0;
        for (; k + 1 < i; k += 2) {
            a0 = O::fms(a0, row[k - i + bw], x[(int64_t)k * stride]);
            a1 = O::fms(a1, row[k + 1 - i + bw], x[(int64_t)(k + 1) * stride]);
        }
        if (k < i) a0 = O::fms(a0, row[k - i + bw], x[(int64_t)k * stride]);
        x[(int64_t)i * stride] = O::fms(a0, O::make(-1.0, 0.0), a1);   // a0 + a1
    }
    // backward: x_i = (y_i - sum_k u_ik x_k) / u_ii
    for (int i = n - 1; i >= 0; --i) {
        const T* row = Bm + (int64_t)i * W;
        const int k1 = min(n - 1, i + bw);
        T a0 = x[(int64_t)i * stride], a1 = O::make(0.0, 0.0);
        int k = i + 1;
        for (; k + 1 <= k1; k += 2) {
            a0 = O::fms(a0, row[k - i + bw], x[(int64_t)k * stride]);
            a1 = O::fms(a1, row[k + 1 - i + bw], x[(int64_t)(k + 1) * stride]);
        }
        if (k <= k1) a0 = O::fms(a0, row[k - i + bw], x[(int64_t)k * stride]);
        x[(int64_t)i * stride] = O::mul(O::fms(a0, O::make(-1.0, 0.0), a1), row[bw]);
    }
}

// The five-point operator with the convection, scale-weighted: (w a / h^2)
// faces, cs = scale c, adv = scale b0; v strided by `stride`.
__device__ __forceinline__ double apply_op(const double* ws, int nx, double cs, double adv,
                                           const double* v, int64_t stride, int i) {
    const int iy = i / nx, ix = i - iy * nx;
    const Faces f = faces(ws, nx, ix, iy);
    const double vi = v[(int64_t)i * stride];
    const double vw = ix > 0 ? v[(int64_t)(i - 1) * stride] : 0.0;
    const double ve = ix < nx - 1 ? v[(int64_t)(i + 1) * stride] : 0.0;
    const double vs = iy > 0 ? v[(int64_t)(i - nx) * stride] : 0.0;
    const double vn = iy < nx - 1 ? v[(int64_t)(i + nx) * stride] : 0.0;
    double acc = cs * vi;
    acc = fma(f.wW, vi - vw, acc);
    acc = fma(f.wE, vi - ve, acc);
    acc = fma(f.wS, vi - vs, acc);
    acc = fma(f.wN, vi - vn, acc);
    acc = fma(adv * (iy + 1), vi - vw, acc);
    acc = fma(adv * (ix + 1), vi - vs, acc);
    return acc;
}

// F by banded solves.  mode 0: item (s, n), start u0 (n = 0) or U[.][n-1],
// J steps, then out[s][i][n] = (I + L_dT) F_i - prev_i, prev = alpha U[.][N-1]
// (n = 0) or U[.][n-1], with L_dT = J L_dt (the jump of the parareal sweep);
// x: scratch [S][n][N].  mode 1: item s, the sequential fine solution,
// out[s][i][n] after every J steps; x: scratch [S][n] (stride 1 per row S).
__global__ void __launch_bounds__(128) k_band_fine(int64_t S, int N, int nx, int J, double dtc,
                                                   double dtf, double adv_dt, double alpha,
                                                   int mode, const double* __restrict__ U,
                                                   const double* __restrict__ u0,
                                                   const double* __restrict__ wdt,
                                                   const double* __restrict__ Bf,
                                                   double* __restrict__ x,
                                                   double* __restrict__ out,
                                                   const int* __restrict__ active) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int n = nx * nx, W = 2 * nx + 1;
    const int64_t items = mode == 0 ? S * N : S;
    if (t >= items) return;
    const int64_t s = mode == 0 ? t / N : t;
    const int n0 = mode == 0 ? (int)(t - s * N) : 0;
    if (!active[s]) return;
    const double* Bm = Bf + s * (int64_t)n * W;
    const double* ws = wdt + s * (int64_t)(2 * nx * (nx + 1));
    double* xs;
    int64_t stride;
    if (mode == 0) {
        xs = x + s * (int64_t)n * N + n0;
        stride = N;
    } else {
        xs = x + s;
        stride = S;
    }
    for (int i = 0; i < n; ++i)
        xs[(int64_t)i * stride] = (mode == 1 || n0 == 0) ? u0[i] : U[(s * n + i) * N + n0 - 1];
    const int nint = mode == 0 ? 1 : N;
    for (int ni = 0; ni < nint; ++ni) {
        for (int j = 0; j < J; ++j) {
            if (dtf != 0.0)
                for (int i = 0; i < n; ++i) xs[(int64_t)i * stride] += dtf;
            band_solve<double>(Bm, nx, xs, stride);
        }
        if (mode == 1)
            for (int i = 0; i < n; ++i) out[(s * n + i) * N + ni] = xs[(int64_t)i * stride];
    }
    if (mode == 0) {
        for (int i = 0; i < n; ++i) {
            const double Fi = xs[(int64_t)i * stride];
            const double LF = J * (apply_op(ws, nx, dtc, adv_dt, xs, stride, i) - dtc * Fi) +
                              J * dtc * Fi;
            const double prev =
                n0 == 0 ? alpha * U[(s * n + i) * N + N - 1] : U[(s * n + i) * N + n0 - 1];
            out[(s * n + i) * N + n0] = (Fi + LF) - prev;
        }
    }
}

// (lambda_k I + L_dT) q = p in place, p: [S][n][K]; one thread per (s, k).
__global__ void __launch_bounds__(128) k_band_cgc(int64_t S, int K, int nx,
                                                  const double2* __restrict__ Bc,
                                                  double2* __restrict__ p,
                                                  const int* __restrict__ active) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * K) return;
    const int64_t s = t / K;
    const int k = (int)(t - s * K);
    if (!active[s]) return;
    const int n = nx * nx, W = 2 * nx + 1;
    band_solve<double2>(Bc + t * (int64_t)n * W, nx, p + s * (int64_t)n * K + k, K);
}

}  // namespace

int64_t band_doubles(int nx) { return (int64_t)nx * nx * (2 * nx + 1); }

void launch_band_factor_fine(int64_t S, int nx, const double* wdt, double dtc, double adv_dt,
                             double* Bf, cudaStream_t st) {
    if (S == 0) return;
    k_band_factor<double><<<(unsigned)((S * 32 + 127) / 128), 128, 0, st>>>(
        S, 1, nx, wdt, dtc, adv_dt, nullptr, Bf);
}

void launch_band_factor_cgc(int64_t S, int K, int nx, const double* wdT, double dTc,
                            double adv_dT, const double2* lam, double2* Bc, cudaStream_t st) {
    if (S == 0) return;
    const int64_t nmat = S * K;
    k_band_factor<double2><<<(unsigned)((nmat * 32 + 127) / 128), 128, 0, st>>>(
        nmat, K, nx, wdT, dTc, adv_dT, lam, Bc);
}

void launch_band_fine(int64_t S, int N, int nx, int J, double dtc, double dtf, double adv_dt,
                      double alpha, int mode, const double* U, const double* u0,
                      const double* wdt, const double* Bf, double* x, double* out,
                      const int* active, cudaStream_t st) {
    const int64_t items = mode == 0 ? S * N : S;
    if (items == 0) return;
    k_band_fine<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(
        S, N, nx, J, dtc, dtf, adv_dt, alpha, mode, U, u0, wdt, Bf, x, out, active);
}

void launch_band_cgc(int64_t S, int K, int nx, const double2* Bc, Cplx<double>* p,
                     const int* active, cudaStream_t st) {
    if (S == 0) return;
    k_band_cgc<<<(unsigned)((S * K + 127) / 128), 128, 0, st>>>(
        S, K, nx, Bc, reinterpret_cast<double2*>(p), active);
}

}  // namespace klecgc
