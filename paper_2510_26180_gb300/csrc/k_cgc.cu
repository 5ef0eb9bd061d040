// Diagonalized coarse grid correction, eq. three steps, with the update and
// the convergence norm (Algorithm 2 step 3):
//   (a) p = F_N^* (Lambda_alpha r)            real DFT along the N coarse times
//   (b) (lambda_k I + dT(A + cI)) q_k = p_k   one complex tridiagonal solve per k
//   (c) u = Lambda_alpha^{-1} F_N q           inverse DFT, fused with the update
//                                             and the per-sample increment norm
// with Lambda_alpha = diag(alpha^{j/N}) and lambda_k = 1 - alpha^{1/N} e^{-2 pi i k/N}.
// (The eigenvector matrix is Lambda_alpha^{-1} F_N: the printed Lambda_alpha F_N
// does not diagonalize C_alpha.)  Real r makes p Hermitian, p_{N-k} = conj(p_k),
// and since A is real the same holds for q, so only k = 0..N/2 are solved.
// The 1/sqrt(N) factors of F_N and F_N^* are combined into one 1/N in (c), and
// the transforms' factors 2 (one each way) into 1/4 there: the inverse scale
// table holds alpha^{-j/N} / (2N).
//
// Layouts: r, U: [S][nx][N]; p, q and the factors: [S][nx][K], K = N/2 + 1.
#include <cmath>

#include "common.cuh"
#include "twiddles.h"

namespace klecgc {

// cos / sin (2 pi t / 128), t in [0, 128), from the first-quadrant literals
// by symmetry.  Every caller passes a compile-time index (fully unrolled
// loops), so each use folds to a literal: no table in memory.
__host__ __device__ constexpr double tw_cos_d(int t) {
    return t <= 32 ? twiddle_cos_q1(t)
         : t <= 64 ? -twiddle_cos_q1(64 - t)
         : t <= 96 ? -twiddle_cos_q1(t - 64)
                   : twiddle_cos_q1(128 - t);
}
__host__ __device__ constexpr double tw_sin_d(int t) {
    return t <= 32 ? twiddle_cos_q1(32 - t)
         : t <= 64 ? twiddle_cos_q1(t - 32)
         : t <= 96 ? -twiddle_cos_q1(96 - t)
                   : -twiddle_cos_q1(t - 96);
}
template <typename T>
__device__ __forceinline__ T tw_cos(int t) { return (T)tw_cos_d(t); }
template <typename T>
__device__ __forceinline__ T tw_sin(int t) { return (T)tw_sin_d(t); }

__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }

template <int L>
__host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1; b < L; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// In-register radix-2 complex FFT of length L (power of 2), unnormalized,
// sign -1 (forward) or +1 (INV).  All indices are compile-time constants.
template <typename T, int L, bool INV>
__device__ __forceinline__ void cfft(T (&re)[L], T (&im)[L]) {
#pragma unroll
    for (int i = 0; i < L; ++i) {
        const int j = bitrev<L>(i);
        if (j > i) {
            T a = re[i]; re[i] = re[j]; re[j] = a;
            T b = im[i]; im[i] = im[j]; im[j] = b;
        }
    }
#pragma unroll
    for (int half = 1; half < L; half *= 2) {
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const int t = k * (kTwiddleN / (2 * half));
            T wr = (T)1, wi = (T)0;
            if (k != 0) {
                wr = tw_cos<T>(t);
                wi = INV ? tw_sin<T>(t) : -tw_sin<T>(t);
            }
#pragma unroll
            for (int b = 0; b < L; b += 2 * half) {
                const int i0 = b + k, i1 = i0 + half;
                if (k == 0 || t == kTwiddleN / 4) {
                    // w = 1, or w = -i (forward) / +i (inverse): a swap and a sign
                    T xr, xi;
                    if (k == 0) {
                        xr = re[i1];
                        xi = im[i1];
                    } else {
                        xr = INV ? -im[i1] : im[i1];
                        xi = INV ? re[i1] : -re[i1];
                    }
                    re[i1] = re[i0] - xr;
                    im[i1] = im[i0] - xi;
                    re[i0] = re[i0] + xr;
                    im[i0] = im[i0] + xi;
                } else {
                    // x0 + w x1 by two FMAs per component, x0 - w x1 = 2 x0 -
                    // (x0 + w x1) by one: six operations where the product
                    // w x1 first and then the sum and difference take eight;
                    // each output is still within a few roundings of
                    // |x0| + |w x1|
                    const T ar = fmat(wr, re[i1], fmat(-wi, im[i1], re[i0]));
                    const T ai = fmat(wr, im[i1], fmat(wi, re[i1], im[i0]));
                    re[i1] = fmat((T)2, re[i0], -ar);
                    im[i1] = fmat((T)2, im[i0], -ai);
                    re[i0] = ar;
                    im[i0] = ai;
                }
            }
        }
    }
}

constexpr int kTX = 32;  // x points per CTA in the transform kernels

// Real DFT of one time series x[0..N-1] (unnormalized, sign -1), times 2,
// into o[0..N/2]: complex FFT of the N/2 packed pairs z_m = x_2m + i x_2m+1,
// then the even/odd split.  With E' = Z_k + conj Z_{L-k} and
// O' = -i (Z_k - conj Z_{L-k}) (twice the even and odd spectra) and
// w = e^{-2 pi i k/N}:  2 X_k = E' + w O'  and  2 X_{L-k} = conj(E' - w O'),
// so one twiddle product serves both outputs of a mirrored pair.  The factor
// 2 (and the inverse's) is removed by the inverse scale table (exact).
template <typename T, int N>
__device__ __forceinline__ void rfft_row(const T (&x)[N], Cplx<T>* o) {
    constexpr int L = N / 2;
    T zr[L], zi[L];
#pragma unroll
    for (int m = 0; m < L; ++m) {
        zr[m] = x[2 * m];
        zi[m] = x[2 * m + 1];
    }
    cfft<T, L, false>(zr, zi);
    // k = 0 and k = L: E' = 2 Re Z_0, O' = 2 Im Z_0, w = 1 and -1
    o[0] = Cplx<T>{(T)2 * (zr[0] + zi[0]), (T)0};
    o[L] = Cplx<T>{(T)2 * (zr[0] - zi[0]), (T)0};
#pragma unroll
    for (int k = 1; k <= L / 2; ++k) {
        const int km = L - k;
        const T Er = zr[k] + zr[km], Ei = zi[k] - zi[km];
        const T Or = zi[k] + zi[km], Oi = zr[km] - zr[k];
        const int t = k * (kTwiddleN / N);
        if (t == kTwiddleN / 4) {   // w = -i
            o[k] = Cplx<T>{Er + Oi, Ei - Or};
            if (km != k) o[km] = Cplx<T>{Er - Oi, -Or - Ei};
        } else {
            // E' + w O' by FMAs, and E' - w O' from it: 2 E' - (E' + w O')
            const T wr = tw_cos<T>(t), wi = -tw_sin<T>(t);
            const T ar = fmat(wr, Or, fmat(-wi, Oi, Er));
            const T ai = fmat(wr, Oi, fmat(wi, Or, Ei));
            o[k] = Cplx<T>{ar, ai};
            if (km != k) o[km] = Cplx<T>{fmat((T)2, Er, -ar), fmat((T)-2, Ei, ai)};
        }
    }
}

// Inverse of rfft_row up to the scale table: X[0..L] (the k <= N/2 half of a
// Hermitian spectrum) to the packed sequence, returned in zr/zi after the
// length-L inverse FFT (4 L (x_2m + i x_2m+1) when X = 2 DFT(x)).
// With E' = X_k + conj X_{L-k}, D' = X_k - conj X_{L-k}, O' = D' e^{+2 pi i k/N}:
// Z'_k = E' + i O' and Z'_{L-k} = conj(E' - i O').
template <typename T, int N>
__device__ __forceinline__ void irfft_row(const Cplx<T>* X, T (&zr)[N / 2], T (&zi)[N / 2]) {
    constexpr int L = N / 2;
    {
        const Cplx<T> A = X[0], B = X[L];
        // k = 0: E' = A + conj B, D' = A - conj B (w = 1)
        const T Er = A.x + B.x, Ei = A.y - B.y, Dr = A.x - B.x, Di = A.y + B.y;
        zr[0] = Er - Di;
        zi[0] = Ei + Dr;
    }
#pragma unroll
    for (int k = 1; k <= L / 2; ++k) {
        const int km = L - k;
        const Cplx<T> A = X[k], B = X[km];
        const T Er = A.x + B.x, Ei = A.y - B.y, Dr = A.x - B.x, Di = A.y + B.y;
        const int t = k * (kTwiddleN / N);
        if (t == kTwiddleN / 4) {   // w = +i: O' = i D'
            zr[k] = Er - Dr;
            zi[k] = Ei - Di;
            if (km != k) {
                zr[km] = Er + Dr;
                zi[km] = -Di - Ei;
            }
        } else {
            // E' + i O' by FMAs, and conj(E' - i O') from it
            const T wr = tw_cos<T>(t), wi = tw_sin<T>(t);
            const T ar = fmat(-wi, Dr, fmat(-wr, Di, Er));
            const T ai = fmat(wr, Dr, fmat(-wi, Di, Ei));
            zr[k] = ar;
            zi[k] = ai;
            if (km != k) {
                zr[km] = fmat((T)2, Er, -ar);
                zi[km] = fmat((T)-2, Ei, ai);
            }
        }
    }
    cfft<T, L, true>(zr, zi);
}

// (a) for the defect path, fused with the accumulation of F and the defect:
//   F_new = F_old + fout (pairs), D = F_new - U (pairs -> float),
//   d = (I + dT(A + cI)) D (flux form, FP32), then p = DFT_n(alpha^{n/N} d).
// The tile carries one halo row on each side for the x-neighbours of D.
// F_new is written to a second buffer: the halo rows are recomputed here and
// written by the neighbouring tile, so an in-place update would race.
constexpr int kTXF = 64;  // x points (= threads) per CTA in the FP32 transform kernels

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// The transform and solve kernels are thin wrappers around per-tile device
// bodies that take their sample and tile and a shared-memory buffer: the
// same bodies serve the persistent stage kernels of the uneven batch, which
// pick the tile from a work queue and carve the buffer from one dynamic
// allocation (static arrays in each instantiation would add up).

template <int N>
__host__ __device__ constexpr size_t fwd_df_smem() {
    return align16((kTXF + 2) * (N + 1) * sizeof(float) + (kTXF + 1) * sizeof(float)) +
           kTXF * (N / 2 + 1) * sizeof(Cplx<float>);
}

template <int N>
__device__ __forceinline__ void fwd_df_tile(
    int64_t s, int x0, int nx, const float* __restrict__ fout, float2* __restrict__ Facc0,
    float2* __restrict__ Facc1, int kit, const float2* __restrict__ Udf,
    const double* __restrict__ wT, float dTreact, const float* __restrict__ scale,
    Cplx<float>* __restrict__ p, char* smem) {
    constexpr int K = N / 2 + 1;
    // iteration k reads F(U^{k-1}) from buffer (k - 1) & 1 (none at k = 0)
    // and writes F(U^k) to buffer k & 1
    const float2* __restrict__ Facc_in = kit == 0 ? nullptr : ((kit & 1) ? Facc0 : Facc1);
    float2* __restrict__ Facc_out = (kit & 1) ? Facc1 : Facc0;
    float (*sD)[N + 1] = reinterpret_cast<float (*)[N + 1]>(smem);
    float* sw = reinterpret_cast<float*>(smem + (kTXF + 2) * (N + 1) * sizeof(float));
    Cplx<float>* sout = reinterpret_cast<Cplx<float>*>(
        smem + align16((kTXF + 2) * (N + 1) * sizeof(float) + (kTXF + 1) * sizeof(float)));
    const int rows = min(kTXF, nx - x0);
    const int tid = threadIdx.x;
    const int64_t base = s * (int64_t)nx * N;
    if constexpr (N % 4 == 0) {
        // 4 consecutive coarse times per access: 16-byte fout, 2 x 16-byte pair loads
        constexpr int G = N / 4;
#pragma unroll 4
        for (int e = tid; e < (rows + 2) * G; e += kTXF) {
            const int row = e / G, c = (e - row * G) * 4, x = x0 - 1 + row;
            float D[4] = {0.f, 0.f, 0.f, 0.f};
            if (x >= 0 && x < nx) {
                const int64_t o = base + (int64_t)x * N + c;
                const float4 f = *reinterpret_cast<const float4*>(fout + o);
                const float4 u01 = *reinterpret_cast<const float4*>(Udf + o);
                const float4 u23 = *reinterpret_cast<const float4*>(Udf + o + 2);
                float2 F0 = make_float2(f.x, 0.f), F1 = make_float2(f.y, 0.f);
                float2 F2 = make_float2(f.z, 0.f), F3 = make_float2(f.w, 0.f);
                if (Facc_in) {
                    const float4 a01 = *reinterpret_cast<const float4*>(Facc_in + o);
                    const float4 a23 = *reinterpret_cast<const float4*>(Facc_in + o + 2);
                    F0 = df_add(make_float2(a01.x, a01.y), f.x);
                    F1 = df_add(make_float2(a01.z, a01.w), f.y);
                    F2 = df_add(make_float2(a23.x, a23.y), f.z);
                    F3 = df_add(make_float2(a23.z, a23.w), f.w);
                }
                if (row >= 1 && row <= rows) {
                    *reinterpret_cast<float4*>(Facc_out + o) = make_float4(F0.x, F0.y, F1.x, F1.y);
                    *reinterpret_cast<float4*>(Facc_out + o + 2) = make_float4(F2.x, F2.y, F3.x, F3.y);
                }
                D[0] = df_sub(F0, make_float2(u01.x, u01.y));
                D[1] = df_sub(F1, make_float2(u01.z, u01.w));
                D[2] = df_sub(F2, make_float2(u23.x, u23.y));
                D[3] = df_sub(F3, make_float2(u23.z, u23.w));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) sD[row][c + q] = D[q];
        }
    } else {
        for (int e = tid; e < (rows + 2) * N; e += kTXF) {
            const int row = e / N, col = e - row * N, x = x0 - 1 + row;
            float D = 0.f;
            if (x >= 0 && x < nx) {
                const int64_t o = base + (int64_t)x * N + col;
                const float f = fout[o];
                const float2 F = Facc_in ? df_add(Facc_in[o], f) : make_float2(f, 0.f);
                if (row >= 1 && row <= rows) Facc_out[o] = F;
                D = df_sub(F, Udf[o]);
            }
            sD[row][col] = D;
        }
    }
    for (int e = tid; e <= rows; e += kTXF) sw[e] = (float)wT[s * (nx + 1) + x0 + e];
    __syncthreads();
    if (tid < rows) {
        const float wl = sw[tid], wr = sw[tid + 1];
        float xs[N];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float D = sD[tid + 1][n];
            const float d = D + wl * (D - sD[tid][n]) - wr * (sD[tid + 2][n] - D) + dTreact * D;
            xs[n] = d * scale[n];
        }
        rfft_row<float, N>(xs, sout + tid * K);
    }
    __syncthreads();
    Cplx<float>* pout = p + (s * nx + x0) * (int64_t)K;
    for (int e = tid; e < rows * K; e += kTXF) pout[e] = sout[e];
}

template <int N>
__global__ void __launch_bounds__(kTXF) k_cgc_forward_df(
    int64_t S, int nx, const float* __restrict__ fout, float2* __restrict__ Facc0,
    float2* __restrict__ Facc1, int k_host, const int* __restrict__ kdev,
    const float2* __restrict__ Udf, const double* __restrict__ wT, float dTreact,
    const float* __restrict__ scale, Cplx<float>* __restrict__ p,
    const int* __restrict__ active) {
    __shared__ __align__(16) char smem[fwd_df_smem<N>()];
    const int64_t s = blockIdx.x;
    if (!active[s]) return;
    fwd_df_tile<N>(s, blockIdx.y * kTXF, nx, fout, Facc0, Facc1, kdev ? *kdev : k_host, Udf, wT,
                   dTreact, scale, p, smem);
}

// (a) for the mixed path (FP32 fine propagator; CGC, update and norms in
// FP64).  The CGC right-hand side is kept in FP64, pre-scaled by the step (a)
// weights: rs_n = alpha^{n/N} r_n.
//   first iteration (c32 == nullptr): r_n = (I + dT(A + cI)) F_n - prev_n with
//     F = fout (F of the start values, FP32 storage), prev_0 = alpha U_{N-1},
//     prev_n = U_{n-1}, formed in FP64;
//   later iterations: F is affine, F(U^k_{n-1}) - F(U^{k-1}_{n-1}) = F0(c_{n-1})
//     with c = U^k - U^{k-1} and fout = F0(c_{n-1}), so
//       r^k_n - r^{k-1}_n = (I + dT(A + cI)) F0(c_{n-1}) - c_{n-1}  (c_{-1} := alpha c_{N-1}),
//     an increment formed in FP32 flux form from the FP32 values it is made
//     of and added to rs in FP64.
// Then p = DFT_n(rs) (times 2, see rfft_row).  rs is updated in place (no
// halo on rs); the halo rows of fout give the x-neighbours of the flux.
template <int N>
__host__ __device__ constexpr size_t fwd_acc_smem() {
    return align16((kTX + 2) * (N + 1) * sizeof(float)) + (kTX + 1) * sizeof(double);
}

template <int N>
__device__ __forceinline__ void fwd_acc_tile(
    int64_t s, int x0, int nx, const float* __restrict__ fout, const float* __restrict__ c32,
    const double* __restrict__ U, const double* __restrict__ wT, double dTreact, double alpha,
    const double* __restrict__ scale, const float* __restrict__ scale32, double* __restrict__ rs,
    Cplx<double>* __restrict__ p, char* smem) {
    constexpr int K = N / 2 + 1;
    // fout rows x0-1 .. x0+rows (the x-neighbours of the flux form); every
    // other row a thread touches is its own and is accessed directly
    float (*sF)[N + 1] = reinterpret_cast<float (*)[N + 1]>(smem);
    double* sw = reinterpret_cast<double*>(smem + align16((kTX + 2) * (N + 1) * sizeof(float)));
    const bool first = c32 == nullptr;
    const int rows = min(kTX, nx - x0);
    const int tid = threadIdx.x;
    const int64_t base = s * (int64_t)nx * N;
    for (int e = tid; e < (rows + 2) * N; e += kTX) {
        const int row = e / N, col = e - row * N, x = x0 - 1 + row;
        sF[row][col] = (x >= 0 && x < nx) ? fout[base + (int64_t)x * N + col] : 0.f;
    }
    for (int e = tid; e <= rows; e += kTX) sw[e] = wT[s * (nx + 1) + x0 + e];
    __syncthreads();
    if (tid >= rows) return;
    const int64_t row = s * (int64_t)nx + x0 + tid;
    const double wl = sw[tid], wr = sw[tid + 1];
    double xs[N];
    if (first) {
        const double* Ur = U + row * N;
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const double F = sF[tid + 1][n];
            const double Fm = sF[tid][n], Fp = sF[tid + 2][n];
            const double prev = n == 0 ? alpha * Ur[N - 1] : Ur[n - 1];
            const double r = F + wl * (F - Fm) - wr * (Fp - F) + dTreact * F;
            xs[n] = scale[n] * (r - prev);
        }
    } else {
        const float* cr = c32 + row * N;
        const double* rr = rs + row * N;
        const float wlf = (float)wl, wrf = (float)wr, rf = (float)dTreact;
        const float af = (float)alpha;
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float D = sF[tid + 1][n];
            const float prev = n == 0 ? af * cr[N - 1] : cr[n - 1];
            const float d = D + wlf * (D - sF[tid][n]) - wrf * (sF[tid + 2][n] - D) + rf * D - prev;
            xs[n] = rr[n] + (double)(scale32[n] * d);
        }
    }
    double* rw = rs + row * N;
#pragma unroll
    for (int n = 0; n < N; ++n) rw[n] = xs[n];
    rfft_row<double, N>(xs, p + row * K);
}

template <int N>
__global__ void __launch_bounds__(kTX) k_cgc_forward_acc(
    int64_t S, int nx, const float* __restrict__ fout, const float* __restrict__ c32,
    const double* __restrict__ U, const double* __restrict__ wT, double dTreact, double alpha,
    const double* __restrict__ scale, const float* __restrict__ scale32, double* __restrict__ rs,
    Cplx<double>* __restrict__ p, const int* __restrict__ active) {
    __shared__ __align__(16) char smem[fwd_acc_smem<N>()];
    const int64_t s = blockIdx.x;
    if (!active[s]) return;
    fwd_acc_tile<N>(s, blockIdx.y * kTX, nx, fout, c32, U, wT, dTreact, alpha, scale, scale32, rs,
                    p, smem);
}

#define KLECGC_N_SWITCH(N, CALL)      \
    switch (N) {                      \
        case 2: CALL(2); break;       \
        case 4: CALL(4); break;       \
        case 8: CALL(8); break;       \
        case 16: CALL(16); break;     \
        case 32: CALL(32); break;     \
        case 64: CALL(64); break;     \
        default: break;               \
    }

void launch_cgc_forward_df(int64_t S, int N, int nx, const float* fout, float2* Facc0,
                           float2* Facc1, int k, const int* kdev, const float2* Udf,
                           const double* wT, double dTreact, const float* scale, Cplx<float>* p,
                           const int* active, cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((nx + kTXF - 1) / kTXF));
#define KLECGC_FDF(NN)                                                                          \
    k_cgc_forward_df<NN><<<grid, kTXF, 0, st>>>(S, nx, fout, Facc0, Facc1, k, kdev, Udf, wT,   \
                                               (float)dTreact, scale, p, active)
    KLECGC_N_SWITCH(N, KLECGC_FDF)
#undef KLECGC_FDF
}

void launch_cgc_forward_acc(int64_t S, int N, int nx, const float* fout, const float* c32,
                            const double* U, const double* wT, double dTreact, double alpha,
                            const double* scale, const float* scale32, double* rs,
                            Cplx<double>* p, const int* active, cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((nx + kTX - 1) / kTX));
#define KLECGC_FACC(NN)                                                                       \
    k_cgc_forward_acc<NN><<<grid, kTX, 0, st>>>(S, nx, fout, c32, U, wT, dTreact, alpha, scale, \
                                                scale32, rs, p, active)
    KLECGC_N_SWITCH(N, KLECGC_FACC)
#undef KLECGC_FACC
}

// (a): thread x transforms its own time series (the row r[s][x][.] is
// contiguous, and so is its spectrum row): direct loads and stores, no
// shared memory.
template <typename T, typename TIN, int N>
__global__ void __launch_bounds__(kTX) k_cgc_forward(int64_t S, int nx, const TIN* __restrict__ r,
                                                     const T* __restrict__ scale,
                                                     Cplx<T>* __restrict__ p,
                                                     const int* __restrict__ active) {
    constexpr int K = N / 2 + 1;
    const int64_t s = blockIdx.x;
    if (!active[s]) return;
    const int x = blockIdx.y * kTX + threadIdx.x;
    if (x >= nx) return;
    const int64_t row = s * nx + x;
    const TIN* rin = r + row * N;
    T xs[N];
#pragma unroll
    for (int n = 0; n < N; ++n) xs[n] = (T)rin[n] * scale[n];
    rfft_row<T, N>(xs, p + row * K);
}

template <typename T, typename TIN>
void launch_cgc_forward(int64_t S, int N, int nx, const TIN* r, const T* scale, Cplx<T>* p,
                        const int* active, cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((nx + kTX - 1) / kTX));
    switch (N) {
#define KLECGC_FWD_CASE(NN) \
    case NN: k_cgc_forward<T, TIN, NN><<<grid, kTX, 0, st>>>(S, nx, r, scale, p, active); break;
        KLECGC_FWD_CASE(2)
        KLECGC_FWD_CASE(4)
        KLECGC_FWD_CASE(8)
        KLECGC_FWD_CASE(16)
        KLECGC_FWD_CASE(32)
        KLECGC_FWD_CASE(64)
#undef KLECGC_FWD_CASE
        default: break;
    }
}
template void launch_cgc_forward<double, double>(int64_t, int, int, const double*, const double*,
                                                 Cplx<double>*, const int*, cudaStream_t);
template void launch_cgc_forward<float, float>(int64_t, int, int, const float*, const float*,
                                               Cplx<float>*, const int*, cudaStream_t);

// (b): one thread per (sample, k); forward sweep w_i = dinv_i (p_i + wT_i w_{i-1}),
// back substitution q_i = w_i - lu_i q_{i+1}, in place.  Rows are loaded in
// chunks of CH before the dependent recurrence runs over them, so that CH
// loads per thread are in flight instead of one.  TW is the type of the face
// weights (FP32 for the FP32 solve: no FP64 conversion in the loop).
template <typename T, typename TW>
__device__ __forceinline__ void cgc_solve_one(int64_t s, int k, int K, int nx,
                                              const Cplx<T>* __restrict__ dinv,
                                              const Cplx<T>* __restrict__ lu,
                                              const TW* __restrict__ wT,
                                              Cplx<T>* __restrict__ p) {
    // rows per load batch (swept 4, 8, 16: 1.049, 1.093, 1.082 ms per
    // launch at 4096 samples; the results do not depend on it)
    constexpr int CH = 4;
    const int64_t base = s * (int64_t)nx * K + k;
    const TW* w = wT + s * (nx + 1);
    T wr = 0, wi = 0;
    for (int i0 = 0; i0 < nx; i0 += CH) {
        Cplx<T> pc[CH], dc[CH];
        T wc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = i0 + c;
            if (i < nx) {
                const int64_t o = base + (int64_t)i * K;
                pc[c] = p[o];
                dc[c] = dinv[o];
                wc[c] = (T)w[i];
            }
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = i0 + c;
            if (i < nx) {
                const T ar = pc[c].x + wc[c] * wr, ai = pc[c].y + wc[c] * wi;
                wr = dc[c].x * ar - dc[c].y * ai;
                wi = dc[c].x * ai + dc[c].y * ar;
                p[base + (int64_t)i * K] = Cplx<T>{wr, wi};
            }
        }
    }
    T qr = 0, qi = 0;
    const int last0 = ((nx - 1) / CH) * CH;
    for (int i0 = last0; i0 >= 0; i0 -= CH) {
        Cplx<T> wc[CH], uc[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int i = i0 + c;
            if (i < nx) {
                const int64_t o = base + (int64_t)i * K;
                wc[c] = p[o];
                uc[c] = lu[o];
            }
        }
#pragma unroll
        for (int c = CH - 1; c >= 0; --c) {
            const int i = i0 + c;
            if (i < nx) {
                const T nr = wc[c].x - (uc[c].x * qr - uc[c].y * qi);
                const T ni = wc[c].y - (uc[c].x * qi + uc[c].y * qr);
                qr = nr;
                qi = ni;
                p[base + (int64_t)i * K] = Cplx<T>{qr, qi};
            }
        }
    }
}

template <typename T, typename TW>
__global__ void __launch_bounds__(128) k_cgc_solve(int64_t S, int K, int nx,
                                                   const Cplx<T>* __restrict__ dinv,
                                                   const Cplx<T>* __restrict__ lu,
                                                   const TW* __restrict__ wT,
                                                   Cplx<T>* __restrict__ p,
                                                   const int* __restrict__ active) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * K) return;
    int64_t s = t / K;
    int k = (int)(t - s * K);
    if (!active[s]) return;
    cgc_solve_one<T, TW>(s, k, K, nx, dinv, lu, wT, p);
}

template <typename T, typename TW>
void launch_cgc_solve(int64_t S, int K, int nx, const Cplx<T>* dinv, const Cplx<T>* lu,
                      const TW* wT, Cplx<T>* p, const int* active, cudaStream_t st) {
    int64_t n = S * K;
    if (n == 0) return;
    k_cgc_solve<T, TW><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(S, K, nx, dinv, lu, wT, p,
                                                                     active);
}
template void launch_cgc_solve<double, double>(int64_t, int, int, const Cplx<double>*,
                                               const Cplx<double>*, const double*, Cplx<double>*,
                                               const int*, cudaStream_t);
template void launch_cgc_solve<float, float>(int64_t, int, int, const Cplx<float>*,
                                             const Cplx<float>*, const float*, Cplx<float>*,
                                             const int*, cudaStream_t);

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}

// (c) + update + increment norm.  Thread x of the tile transforms its own
// spectrum row, read directly (read-only, contiguous); U and the FP32
// increments pass through shared memory so that their global reads and
// writes are coalesced (a thread's own rows read and written in place would
// serialize each load behind the store before it).
// mode 0: U = u, c32 = u - U_old, delta = max |u - U_old|;
// mode 1: U += u, c32 = u, delta = max |u|;  mode 2: U = u.
template <int N>
__host__ __device__ constexpr size_t inv_smem() {
    return align16(kTX * (N + 1) * sizeof(double)) + kTX * (N + 1) * sizeof(float);
}

template <typename T, int N>
__device__ __forceinline__ void inv_tile(int64_t s, int x0, int nx, const Cplx<T>* __restrict__ q,
                                         const T* __restrict__ iscale, double* __restrict__ U,
                                         int mode, unsigned long long* __restrict__ delta,
                                         float* __restrict__ c32, char* smem) {
    constexpr int L = N / 2, K = N / 2 + 1;
    double (*su)[N + 1] = reinterpret_cast<double (*)[N + 1]>(smem);
    float (*sc)[N + 1] = reinterpret_cast<float (*)[N + 1]>(smem + align16(kTX * (N + 1) * sizeof(double)));
    const int rows = min(kTX, nx - x0);
    const int tid = threadIdx.x;
    double* Ut = U + (s * nx + x0) * (int64_t)N;
    if (mode != 2)
        for (int e = tid; e < rows * N; e += kTX) {
            const int row = e / N, col = e - row * N;
            su[row][col] = Ut[e];
        }
    __syncthreads();
    unsigned long long dmax = 0ull;
    if (tid < rows) {
        T zr[L], zi[L];
        irfft_row<T, N>(q + (s * nx + x0 + tid) * (int64_t)K, zr, zi);
#pragma unroll
        for (int m = 0; m < L; ++m) {
            const double u0 = (double)(zr[m] * iscale[2 * m]);
            const double u1 = (double)(zi[m] * iscale[2 * m + 1]);
            if (mode == 0) {
                const double c0 = u0 - su[tid][2 * m], c1 = u1 - su[tid][2 * m + 1];
                dmax = max(dmax, abs_bits(c0));
                dmax = max(dmax, abs_bits(c1));
                sc[tid][2 * m] = (float)c0;
                sc[tid][2 * m + 1] = (float)c1;
                su[tid][2 * m] = u0;
                su[tid][2 * m + 1] = u1;
            } else if (mode == 1) {
                dmax = max(dmax, abs_bits(u0));
                dmax = max(dmax, abs_bits(u1));
                sc[tid][2 * m] = (float)u0;
                sc[tid][2 * m + 1] = (float)u1;
                su[tid][2 * m] += u0;
                su[tid][2 * m + 1] += u1;
            } else {
                su[tid][2 * m] = u0;
                su[tid][2 * m + 1] = u1;
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < rows * N; e += kTX) {
        const int row = e / N, col = e - row * N;
        Ut[e] = su[row][col];
    }
    if (mode != 2 && c32) {
        float* ct = c32 + (s * nx + x0) * (int64_t)N;
        for (int e = tid; e < rows * N; e += kTX) {
            const int row = e / N, col = e - row * N;
            ct[e] = sc[row][col];
        }
    }
    if (mode != 2) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
        if (tid == 0 && dmax) atomicMax(delta + s, dmax);
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(kTX) k_cgc_inverse(int64_t S, int nx,
                                                     const Cplx<T>* __restrict__ q,
                                                     const T* __restrict__ iscale,
                                                     double* __restrict__ U, int mode,
                                                     unsigned long long* __restrict__ delta,
                                                     float* __restrict__ c32,
                                                     const int* __restrict__ active) {
    __shared__ __align__(16) char smem[inv_smem<N>()];
    const int64_t s = blockIdx.x;
    if (!active[s]) return;
    inv_tile<T, N>(s, blockIdx.y * kTX, nx, q, iscale, U, mode, delta, c32, smem);
}

template <typename T>
void launch_cgc_inverse(int64_t S, int N, int nx, const Cplx<T>* q, const T* iscale, double* U,
                        int mode, unsigned long long* delta, float* c32, const int* active,
                        cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((nx + kTX - 1) / kTX));
    switch (N) {
#define KLECGC_INV_CASE(NN)                                                                 \
    case NN:                                                                                \
        k_cgc_inverse<T, NN><<<grid, kTX, 0, st>>>(S, nx, q, iscale, U, mode, delta, c32, active); \
        break;
        KLECGC_INV_CASE(2)
        KLECGC_INV_CASE(4)
        KLECGC_INV_CASE(8)
        KLECGC_INV_CASE(16)
        KLECGC_INV_CASE(32)
        KLECGC_INV_CASE(64)
#undef KLECGC_INV_CASE
        default: break;
    }
}
template void launch_cgc_inverse<double>(int64_t, int, int, const Cplx<double>*, const double*,
                                         double*, int, unsigned long long*, float*, const int*,
                                         cudaStream_t);
template void launch_cgc_inverse<float>(int64_t, int, int, const Cplx<float>*, const float*,
                                        double*, int, unsigned long long*, float*, const int*,
                                        cudaStream_t);

// (c) + update for the defect path: U (pairs) += u, c32 = u, delta = max|u|.
template <int N>
__host__ __device__ constexpr size_t inv_df_smem() {
    return align16(kTX * 2 * (N / 2 + 1) * sizeof(float)) + kTX * (N + 1) * sizeof(float2);
}

template <int N>
__device__ __forceinline__ void inv_df_tile(int64_t s, int x0, int nx,
                                            const Cplx<float>* __restrict__ q,
                                            const float* __restrict__ iscale,
                                            float2* __restrict__ Udf,
                                            unsigned long long* __restrict__ delta,
                                            float* __restrict__ c32, char* smem) {
    constexpr int L = N / 2, K = N / 2 + 1;
    // The row of q a thread transforms and the row of increments it writes
    // share storage (2K >= N + 1 floats per row): each thread reads its whole
    // q row before it writes its increments, and touches no other row between
    // the barriers; this keeps shared memory at 25 KB per CTA (9 CTAs per SM).
    float* sqc = reinterpret_cast<float*>(smem);
    float2 (*su)[N + 1] = reinterpret_cast<float2 (*)[N + 1]>(smem + align16(kTX * 2 * K * sizeof(float)));
    Cplx<float>* sq = reinterpret_cast<Cplx<float>*>(sqc);   // [kTX][K]
    auto sc = [&](int row, int c) -> float& { return sqc[row * 2 * K + c]; };
    const int rows = min(kTX, nx - x0);
    const int tid = threadIdx.x;
    const Cplx<float>* qin = q + (s * nx + x0) * (int64_t)K;
    for (int e = tid; e < rows * K; e += kTX) sq[e] = qin[e];
    float2* Ut = Udf + (s * nx + x0) * (int64_t)N;
    if constexpr (N % 2 == 0 && N >= 2) {
        constexpr int G = N / 2;
        for (int e = tid; e < rows * G; e += kTX) {
            const int row = e / G, c = (e - row * G) * 2;
            const float4 v = *reinterpret_cast<const float4*>(Ut + (int64_t)row * N + c);
            su[row][c] = make_float2(v.x, v.y);
            su[row][c + 1] = make_float2(v.z, v.w);
        }
    }
    __syncthreads();
    float umax = 0.f;
    bool bad = false;
    if (tid < rows) {
        float zr[L], zi[L];
        irfft_row<float, N>(sq + tid * K, zr, zi);
#pragma unroll
        for (int m = 0; m < L; ++m) {
            const float u0 = zr[m] * iscale[2 * m], u1 = zi[m] * iscale[2 * m + 1];
            umax = fmaxf(umax, fmaxf(fabsf(u0), fabsf(u1)));
            bad |= (u0 != u0) || (u1 != u1);
            su[tid][2 * m] = df_add(su[tid][2 * m], u0);
            su[tid][2 * m + 1] = df_add(su[tid][2 * m + 1], u1);
            sc(tid, 2 * m) = u0;
            sc(tid, 2 * m + 1) = u1;
        }
    }
    __syncthreads();
    float* ct = c32 + (s * nx + x0) * (int64_t)N;
    {
        constexpr int G = N / 2;
        for (int e = tid; e < rows * G; e += kTX) {
            const int row = e / G, c = (e - row * G) * 2;
            const float2 a = su[row][c], b = su[row][c + 1];
            *reinterpret_cast<float4*>(Ut + (int64_t)row * N + c) = make_float4(a.x, a.y, b.x, b.y);
            *reinterpret_cast<float2*>(ct + (int64_t)row * N + c) = make_float2(sc(row, c), sc(row, c + 1));
        }
    }
    // a NaN increment must reach the stopping rule (fmaxf drops NaNs)
    unsigned long long dmax = bad ? 0x7ff8000000000000ull : abs_bits((double)umax);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    if ((tid & 31) == 0 && dmax) atomicMax(delta + s, dmax);
}

template <int N>
__global__ void __launch_bounds__(kTX) k_cgc_inverse_df(int64_t S, int nx,
                                                         const Cplx<float>* __restrict__ q,
                                                         const float* __restrict__ iscale,
                                                         float2* __restrict__ Udf,
                                                         unsigned long long* __restrict__ delta,
                                                         float* __restrict__ c32,
                                                         const int* __restrict__ active) {
    __shared__ __align__(16) char smem[inv_df_smem<N>()];
    const int64_t s = blockIdx.x;
    if (!active[s]) return;
    inv_df_tile<N>(s, blockIdx.y * kTX, nx, q, iscale, Udf, delta, c32, smem);
}

void launch_cgc_inverse_df(int64_t S, int N, int nx, const Cplx<float>* q, const float* iscale,
                           float2* Udf, unsigned long long* delta, float* c32, const int* active,
                           cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((nx + kTX - 1) / kTX));
#define KLECGC_IDF(NN) \
    k_cgc_inverse_df<NN><<<grid, kTX, 0, st>>>(S, nx, q, iscale, Udf, delta, c32, active)
    KLECGC_N_SWITCH(N, KLECGC_IDF)
#undef KLECGC_IDF
}

__global__ void k_to_pairs(double* __restrict__ U, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double v = U[t];
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    reinterpret_cast<float2*>(U)[t] = make_float2(hi, lo);
}

void launch_to_pairs(double* U, int64_t n, cudaStream_t st) {
    if (n == 0) return;
    k_to_pairs<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(U, n);
}

__global__ void k_pairs_transpose_out(const float2* __restrict__ in, double* __restrict__ out,
                                      int A, int B) {
    __shared__ double tile[32][33];
    const int64_t s = blockIdx.x;
    const float2* src = in + s * (int64_t)A * B;
    double* dst = out + s * (int64_t)A * B;
    int a0 = blockIdx.y * 32, b0 = blockIdx.z * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int a = a0 + y, b = b0 + threadIdx.x;
        if (a < A && b < B) {
            const float2 v = src[(int64_t)a * B + b];
            tile[y][threadIdx.x] = (double)v.x + (double)v.y;
        }
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int b = b0 + y, a = a0 + threadIdx.x;
        if (a < A && b < B) dst[(int64_t)b * A + a] = tile[threadIdx.x][y];
    }
}

void launch_pairs_transpose_out(const float2* in, double* out, int64_t S, int nx, int N,
                                cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((nx + 31) / 32), (unsigned)((N + 31) / 32));
    k_pairs_transpose_out<<<grid, dim3(32, 8), 0, st>>>(in, out, nx, N);
}

// Stopping rule per sample (Algorithm 2, Step 3): stop after the first
// iteration whose increment max-norm is <= tol.
__global__ void k_convergence(int64_t S, int iter_host, const int* __restrict__ kdev, int kmax,
                              double tol, unsigned long long* __restrict__ delta,
                              int* __restrict__ active, int32_t* __restrict__ iters,
                              int32_t* __restrict__ status, int* __restrict__ n_active) {
    const int iter = kdev ? *kdev : iter_host;
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool still = false;
    if (s < S && active[s]) {
        double d = __longlong_as_double((long long)delta[s]);
        delta[s] = 0ull;
        if (!isfinite(d)) {
            active[s] = 0;
            iters[s] = -2;
            status[s] = 4;  // KLECGC_E_NONFINITE
        } else if (d <= tol) {
            active[s] = 0;
            iters[s] = iter + 1;
            status[s] = 0;
        } else if (iter + 1 >= kmax) {
            active[s] = 0;
            iters[s] = -1;
            status[s] = 3;  // KLECGC_E_NOT_CONVERGED
        } else {
            still = true;
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, still);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_active, __popc(b));
}

void launch_convergence(int64_t S, int iter, int kmax, double tol, unsigned long long* delta,
                        int* active, int32_t* iters, int32_t* status, int* n_active,
                        cudaStream_t st, const int* kdev) {
    if (S == 0) return;
    k_convergence<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(S, iter, kdev, kmax, tol, delta,
                                                                active, iters, status, n_active);
}

// End of one iteration of a device-driven parareal loop (the body of a CUDA
// graph WHILE node): the iteration counter advances, and the loop continues
// while some sample is active and fewer than kmax iterations have run.
__global__ void k_loop_tail(int* __restrict__ kdev, const int* __restrict__ n_active, int kmax,
                            cudaGraphConditionalHandle handle) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int k = *kdev + 1;
        *kdev = k;
        cudaGraphSetConditional(handle, (*n_active > 0 && k < kmax) ? 1u : 0u);
    }
}

void launch_loop_tail(int* kdev, const int* n_active, int kmax, cudaGraphConditionalHandle h,
                      cudaStream_t st) {
    k_loop_tail<<<1, 32, 0, st>>>(kdev, n_active, kmax, h);
}

__global__ void k_set_int(int* p, int v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

void launch_set_int(int* p, int v, cudaStream_t st) { k_set_int<<<1, 32, 0, st>>>(p, v); }

__global__ void k_transpose(const double* __restrict__ in, double* __restrict__ out, int A, int B) {
    __shared__ double tile[32][33];
    const int64_t s = blockIdx.x;
    const double* src = in + s * (int64_t)A * B;
    double* dst = out + s * (int64_t)A * B;
    int a0 = blockIdx.y * 32, b0 = blockIdx.z * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int a = a0 + y, b = b0 + threadIdx.x;
        if (a < A && b < B) tile[y][threadIdx.x] = src[(int64_t)a * B + b];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int b = b0 + y, a = a0 + threadIdx.x;
        if (a < A && b < B) dst[(int64_t)b * A + a] = tile[threadIdx.x][y];
    }
}

void launch_transpose(const double* in, double* out, int64_t S, int A, int B, cudaStream_t st) {
    if (S == 0) return;
    dim3 grid((unsigned)S, (unsigned)((A + 31) / 32), (unsigned)((B + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, out, A, B);
}

}  // namespace klecgc

// ---- the uneven batch: persistent stage kernels over all classes
namespace klecgc {

// Thread 0 takes the next task index; every thread of the CTA returns it.
__device__ __forceinline__ int batch_next(int* queue, int* s_task) {
    if (threadIdx.x == 0) *s_task = atomicAdd(queue, 1);
    __syncthreads();
    const int t = *s_task;
    __syncthreads();
    return t;
}

// (a): tiles of kTX rows (MIXED, FP64 transform of the accumulated right-hand
// side) or kTXF rows (MIXED_DEFECT, FP32 defect transform).
template <int DEFECT>
__global__ void __launch_bounds__(DEFECT ? kTXF : kTX) k_batch_fwd(
    const BatchClass* __restrict__ cls, const BatchTask* __restrict__ tasks, int ntasks,
    int* queue, int k_host, const int* __restrict__ kdev) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_task;
    const int k = kdev ? *kdev : k_host;
    for (;;) {
        const int t = batch_next(queue, &s_task);
        if (t >= ntasks) break;
        const BatchTask tk = tasks[t];
        const BatchClass& C = cls[tk.c];
        if (!C.active[tk.s]) continue;
        if (DEFECT) {
            const int x0 = tk.part * kTXF;
#define KLECGC_BF(NN)                                                                          \
    fwd_df_tile<NN>(tk.s, x0, C.nx, C.fout, C.Facc0, C.Facc1, k, C.Udf, C.wT, (float)C.dTreact, \
                    C.sc32, C.p32, smem)
            KLECGC_N_SWITCH(C.N, KLECGC_BF)
#undef KLECGC_BF
        } else {
            const int x0 = tk.part * kTX;
            const float* c = k == 0 ? nullptr : C.c32;
#define KLECGC_BA(NN)                                                                          \
    fwd_acc_tile<NN>(tk.s, x0, C.nx, C.fout, c, C.U, C.wT, C.dTreact, C.alpha, C.sc64, C.sc32, \
                     C.rs, C.p64, smem)
            KLECGC_N_SWITCH(C.N, KLECGC_BA)
#undef KLECGC_BA
        }
        __syncthreads();
    }
}

// (b): chunks of 128 consecutive (sample, k) systems of one class.
template <int DEFECT>
__global__ void __launch_bounds__(128) k_batch_solve(const BatchClass* __restrict__ cls,
                                                     const BatchTask* __restrict__ tasks,
                                                     int ntasks, int* queue) {
    __shared__ int s_task;
    for (;;) {
        const int t = batch_next(queue, &s_task);
        if (t >= ntasks) break;
        const BatchTask tk = tasks[t];
        const BatchClass& C = cls[tk.c];
        const int64_t sys = (int64_t)tk.part + threadIdx.x;
        if (sys < C.S * C.K) {
            const int64_t s = sys / C.K;
            const int kk = (int)(sys - s * C.K);
            if (C.active[s]) {
                if (DEFECT)
                    cgc_solve_one<float, float>(s, kk, C.K, C.nx, C.dinv32, C.lu32, C.wT32, C.p32);
                else
                    cgc_solve_one<double, double>(s, kk, C.K, C.nx, C.dinv64, C.lu64, C.wT, C.p64);
            }
        }
    }
}

// (c) + update + increment norm: tiles of kTX rows.
template <int DEFECT>
__global__ void __launch_bounds__(kTX) k_batch_inv(const BatchClass* __restrict__ cls,
                                                   const BatchTask* __restrict__ tasks, int ntasks,
                                                   int* queue) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_task;
    for (;;) {
        const int t = batch_next(queue, &s_task);
        if (t >= ntasks) break;
        const BatchTask tk = tasks[t];
        const BatchClass& C = cls[tk.c];
        if (!C.active[tk.s]) continue;
        const int x0 = tk.part * kTX;
        if (DEFECT) {
#define KLECGC_BI(NN) inv_df_tile<NN>(tk.s, x0, C.nx, C.p32, C.isc32, C.Udf, C.delta, C.c32, smem)
            KLECGC_N_SWITCH(C.N, KLECGC_BI)
#undef KLECGC_BI
        } else {
#define KLECGC_BI(NN) \
    inv_tile<double, NN>(tk.s, x0, C.nx, C.p64, C.isc64, C.U, 0, C.delta, C.c32, smem)
            KLECGC_N_SWITCH(C.N, KLECGC_BI)
#undef KLECGC_BI
        }
        __syncthreads();
    }
}

// Stopping rule (Algorithm 2, Step 3) for every instance of the batch.
__global__ void k_batch_conv(const BatchClass* __restrict__ cls, const BatchTask* __restrict__ inst,
                             int64_t n, int k_host, const int* __restrict__ kdev,
                             int* __restrict__ n_active) {
    const int iter = kdev ? *kdev : k_host;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool still = false;
    if (i < n) {
        const BatchTask tk = inst[i];
        const BatchClass& C = cls[tk.c];
        const int64_t s = tk.s;
        if (C.active[s]) {
            const double d = __longlong_as_double((long long)C.delta[s]);
            C.delta[s] = 0ull;
            if (!isfinite(d)) {
                C.active[s] = 0;
                C.iters[s] = -2;
                C.status[s] = 4;  // KLECGC_E_NONFINITE
            } else if (d <= C.tol) {
                C.active[s] = 0;
                C.iters[s] = iter + 1;
                C.status[s] = 0;
            } else if (iter + 1 >= C.kmax) {
                C.active[s] = 0;
                C.iters[s] = -1;
                C.status[s] = 3;  // KLECGC_E_NOT_CONVERGED
            } else {
                still = true;
            }
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, still);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_active, __popc(b));
}

int batch_transform_tile(int defect) { return defect ? kTXF : kTX; }

static size_t batch_fwd_smem(int defect) {
    return defect ? fwd_df_smem<64>() : fwd_acc_smem<64>();
}
static size_t batch_inv_smem(int defect) { return defect ? inv_df_smem<64>() : inv_smem<64>(); }

int batch_grid(int kind, int defect) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    if (kind == 0) {
        if (defect) {
            cudaFuncSetAttribute(k_batch_fwd<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch_fwd_smem(1));
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_fwd<1>, kTXF,
                                                              batch_fwd_smem(1));
        } else {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_fwd<0>, kTX,
                                                              batch_fwd_smem(0));
        }
    } else if (kind == 1) {
        e = defect ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_solve<1>, 128, 0)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_solve<0>, 128, 0);
    } else {
        e = defect ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_inv<1>, kTX,
                                                                   batch_inv_smem(1))
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_inv<0>, kTX,
                                                                   batch_inv_smem(0));
    }
    if (e != cudaSuccess || per < 1) per = 1;
    return sms * per;
}

void launch_batch_fwd(int defect, const BatchClass* cls, const BatchTask* tasks, int ntasks,
                      int* queue, int k_host, const int* kdev, int grid, cudaStream_t st) {
    if (ntasks == 0) return;
    if (defect)
        k_batch_fwd<1><<<grid, kTXF, batch_fwd_smem(1), st>>>(cls, tasks, ntasks, queue, k_host, kdev);
    else
        k_batch_fwd<0><<<grid, kTX, batch_fwd_smem(0), st>>>(cls, tasks, ntasks, queue, k_host, kdev);
}

void launch_batch_solve(int defect, const BatchClass* cls, const BatchTask* tasks, int ntasks,
                        int* queue, int grid, cudaStream_t st) {
    if (ntasks == 0) return;
    if (defect)
        k_batch_solve<1><<<grid, 128, 0, st>>>(cls, tasks, ntasks, queue);
    else
        k_batch_solve<0><<<grid, 128, 0, st>>>(cls, tasks, ntasks, queue);
}

void launch_batch_inv(int defect, const BatchClass* cls, const BatchTask* tasks, int ntasks,
                      int* queue, int grid, cudaStream_t st) {
    if (ntasks == 0) return;
    if (defect)
        k_batch_inv<1><<<grid, kTX, batch_inv_smem(1), st>>>(cls, tasks, ntasks, queue);
    else
        k_batch_inv<0><<<grid, kTX, batch_inv_smem(0), st>>>(cls, tasks, ntasks, queue);
}

void launch_batch_conv(const BatchClass* cls, const BatchTask* inst, int64_t n, int k_host,
                       const int* kdev, int* n_active, cudaStream_t st) {
    if (n == 0) return;
    k_batch_conv<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cls, inst, n, k_host, kdev, n_active);
}

}  // namespace klecgc
