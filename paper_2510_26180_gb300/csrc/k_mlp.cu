// Learned initial guess: MLP xi -> coarse state at 64
// points per coarse time, its training kernels and the grid maps.
//
// GEMMs run on the tensor cores with BF16 operands and FP32 accumulation
// (warp-level mma.sync m16n8k16).  The network is small (1.19 M parameters,
// <= 8.6 GFLOP per pass at 4096 samples), so these products are latency
// bound and a warp-level MMA serves them; the master weights, Adam moments,
// pre-activations and the loss stay FP32.
#include <cuda_bf16.h>

#include "common.cuh"

namespace klecgc {

namespace {

constexpr int BM = 64, BN = 64, BK = 32, GT = 128;

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// C[m][n] = sum_k A(m,k) B(k,n); A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n].  Epilogue: v = acc (+ bias[n]);
// if zmask: v = zmask[m*ldz+n] > 0 ? v : 0; C (FP32) <- v; Cb (BF16) <- relu ? max(v,0) : v.
template <bool TA, bool TB>
__global__ void __launch_bounds__(GT) k_gemm_bf16(int M, int N, int K,
                                                  const __nv_bfloat16* __restrict__ A, int lda,
                                                  const __nv_bfloat16* __restrict__ B, int ldb,
                                                  const float* __restrict__ bias,
                                                  const float* __restrict__ zmask, int ldz,
                                                  float* __restrict__ C, int ldc,
                                                  __nv_bfloat16* __restrict__ Cb, int ldcb,
                                                  bool relu) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + 8];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += GT) {
            int r, c;
            if (TA) {  // A stored [K][M]: consecutive threads along m
                r = e % BM;
                c = e / BM;
            } else {
                r = e / BK;
                c = e % BK;
            }
            const int gm = m0 + r, gk = k0 + c;
            __nv_bfloat16 v = zero;
            if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[r][c] = v;
        }
        for (int e = tid; e < BN * BK; e += GT) {
            int n, c;
            if (TB) {  // B stored [N][K]: consecutive threads along k
                n = e / BK;
                c = e % BK;
            } else {
                n = e % BN;
                c = e / BN;
            }
            const int gn = n0 + n, gk = k0 + c;
            __nv_bfloat16 v = zero;
            if (gn < N && gk < K) v = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
            Bs[n][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = wm * 32 + mt * 16 + g;
                af[mt][0] = ld_pair(&As[r0][ks + 2 * t]);
                af[mt][1] = ld_pair(&As[r0 + 8][ks + 2 * t]);
                af[mt][2] = ld_pair(&As[r0][ks + 8 + 2 * t]);
                af[mt][3] = ld_pair(&As[r0 + 8][ks + 8 + 2 * t]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = wn * 32 + nt * 8 + g;
                bf[nt][0] = ld_pair(&Bs[n][ks + 2 * t]);
                bf[nt][1] = ld_pair(&Bs[n][ks + 8 + 2 * t]);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]),
                          "+f"(acc[mt][nt][3])
                        : "r"(af[mt][0]), "r"(af[mt][1]), "r"(af[mt][2]), "r"(af[mt][3]),
                          "r"(bf[nt][0]), "r"(bf[nt][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm * 32 + mt * 16 + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn * 32 + nt * 8 + 2 * t + (r & 1);
                if (m >= M || n >= N) continue;
                float v = acc[mt][nt][r];
                if (bias) v += bias[n];
                if (zmask && !(zmask[(int64_t)m * ldz + n] > 0.f)) v = 0.f;
                if (C) C[(int64_t)m * ldc + n] = v;
                if (Cb) Cb[(int64_t)m * ldcb + n] = __float2bfloat16(relu ? fmaxf(v, 0.f) : v);
            }
}

}  // namespace

void launch_gemm_bf16(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16* A, int lda,
                      const __nv_bfloat16* B, int ldb, const float* bias, const float* zmask,
                      int ldz, float* C, int ldc, __nv_bfloat16* Cb, int ldcb, bool relu,
                      cudaStream_t st) {
    if (M == 0 || N == 0) return;
    dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
#define KLECGC_G(TA_, TB_)                                                                     \
    k_gemm_bf16<TA_, TB_><<<grid, GT, 0, st>>>(M, N, K, A, lda, B, ldb, bias, zmask, ldz, C, ldc, \
                                               Cb, ldcb, relu)
    if (!ta && !tb) KLECGC_G(false, false);
    else if (!ta && tb) KLECGC_G(false, true);
    else if (ta && !tb) KLECGC_G(true, false);
    else KLECGC_G(true, true);
#undef KLECGC_G
}

// X batch (BF16) and normalized targets for rows perm[b] (perm may be null).
__global__ void k_mlp_gather(int B, int M, int D, const int* __restrict__ perm, int b0,
                             const double* __restrict__ xi, const float* __restrict__ targ,
                             const float* __restrict__ mean, const float* __restrict__ inv_std,
                             __nv_bfloat16* __restrict__ X, float* __restrict__ T) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nx_ = (int64_t)B * M, nt_ = (int64_t)B * D;
    if (e < nx_) {
        const int b = (int)(e / M), j = (int)(e - (int64_t)b * M);
        const int row = perm ? perm[b0 + b] : b0 + b;
        X[e] = __float2bfloat16((float)xi[(int64_t)row * M + j]);
    }
    if (targ && e < nt_) {
        const int b = (int)(e / D), c = (int)(e - (int64_t)b * D);
        const int row = perm ? perm[b0 + b] : b0 + b;
        T[e] = (targ[(int64_t)row * D + c] - mean[c]) * inv_std[c];
    }
}

void launch_mlp_gather(int B, int M, int D, const int* perm, int b0, const double* xi,
                       const float* targ, const float* mean, const float* inv_std,
                       __nv_bfloat16* X, float* T, cudaStream_t st) {
    const int64_t n = (int64_t)B * (targ ? D : M);
    const int64_t m = (int64_t)B * M > n ? (int64_t)B * M : n;
    k_mlp_gather<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(B, M, D, perm, b0, xi, targ, mean,
                                                              inv_std, X, T);
}

// dY = 2 (Y - T) gscale as FP32 and BF16; loss += sum (Y - T)^2 lscale.
__global__ void k_mse(int64_t n, float gscale, float lscale, const float* __restrict__ Y,
                      const float* __restrict__ T, float* __restrict__ dY,
                      __nv_bfloat16* __restrict__ dYb, float* __restrict__ loss) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float part = 0.f;
    if (e < n) {
        const float r = Y[e] - T[e];
        const float g = 2.f * r * gscale;
        dY[e] = g;
        dYb[e] = __float2bfloat16(g);
        part = r * r * lscale;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0 && part != 0.f) atomicAdd(loss, part);
}

void launch_mse(int64_t n, float gscale, float lscale, const float* Y, const float* T, float* dY,
                __nv_bfloat16* dYb, float* loss, cudaStream_t st) {
    k_mse<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, gscale, lscale, Y, T, dY, dYb, loss);
}

// db[c] = sum_b dZ[b][c]
__global__ void k_colsum(int B, int D, const float* __restrict__ dZ, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * D + c];
    db[c] = s;
}

void launch_colsum(int B, int D, const float* dZ, float* db, cudaStream_t st) {
    k_colsum<<<(unsigned)((D + 127) / 128), 128, 0, st>>>(B, D, dZ, db);
}

// Adam on the flat FP32 parameters; refreshes the BF16 copy used by the GEMMs.
__global__ void k_adam(int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ thb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float w = th[e] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    th[e] = w;
    thb[e] = __float2bfloat16(w);
}

void launch_adam(int64_t n, float lr, int t, float* th, const float* g, float* m, float* v,
                 __nv_bfloat16* thb, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, t)));
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, lr, b1, b2, 1e-8f, c1, c2, th, g, m, v,
                                                        thb);
}

__global__ void k_f32_to_bf16(int64_t n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) y[e] = __float2bfloat16(x[e]);
}

void launch_f32_to_bf16(int64_t n, const float* x, __nv_bfloat16* y, cudaStream_t st) {
    if (n == 0) return;
    k_f32_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y);
}

// [S][N][nx] (caller layout, FP64) -> [S][N][64] at x_m = (m+1)/65 (linear
// interpolation, zero values at x = 0 and 1), FP32.
__global__ void k_downsample(int64_t rows, int nx, const double* __restrict__ U,
                             float* __restrict__ T) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * 64) return;
    const int64_t r = e / 64;
    const int m = (int)(e - r * 64);
    // grid point j has x = j/(nx+1), j = 0..nx+1; row value index j-1
    const double pos = (double)(m + 1) * (nx + 1) / 65.0;
    int j = (int)floor(pos);
    if (j > nx) j = nx;
    const double f = pos - j;
    const double* u = U + r * nx;
    const double a = (j >= 1 && j <= nx) ? u[j - 1] : 0.0;
    const double b = (j + 1 >= 1 && j + 1 <= nx) ? u[j] : 0.0;
    T[e] = (float)(a + f * (b - a));
}

void launch_downsample(int64_t rows, int nx, const double* U, float* T, cudaStream_t st) {
    if (rows == 0) return;
    k_downsample<<<(unsigned)((rows * 64 + 255) / 256), 256, 0, st>>>(rows, nx, U, T);
}

// Network output [S][N*64] (normalized) -> U[s][i][n] (internal layout, FP64):
// de-normalize, then linear interpolation from (0, x_1..x_64, 1) to x_i = (i+1)/(nx+1).
__global__ void k_upsample(int64_t S, int N, int nx, const float* __restrict__ Y,
                           const float* __restrict__ mean, const float* __restrict__ stdv,
                           double* __restrict__ U, int accumulate) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= S * (int64_t)nx * N) return;
    const int n = (int)(e % N);
    const int64_t si = e / N;
    const int i = (int)(si % nx);
    const int64_t s = si / nx;
    const double pos = (double)(i + 1) * 65.0 / (nx + 1);  // in units of the coarse spacing
    int m = (int)floor(pos);                              // between coarse nodes m and m+1
    if (m > 64) m = 64;
    const double f = pos - m;
    const float* y = Y + s * (int64_t)N * 64 + (int64_t)n * 64;
    const float* mu = mean + n * 64;
    const float* sd = stdv + n * 64;
    auto node = [&](int k) -> double {  // value at coarse node k (0 and 65 are the boundary)
        return (k >= 1 && k <= 64) ? (double)(mu[k - 1] + sd[k - 1] * y[k - 1]) : 0.0;
    };
    const double a = node(m), b = node(m + 1);
    const double v = a + f * (b - a);
    U[e] = accumulate ? U[e] + v : v;
}

__global__ void k_sub_f32(int64_t n, float* __restrict__ a, const float* __restrict__ b) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) a[t] -= b[t];
}

void launch_upsample(int64_t S, int N, int nx, const float* Y, const float* mean,
                     const float* stdv, double* U, bool accumulate, cudaStream_t st) {
    const int64_t n = S * (int64_t)nx * N;
    if (n == 0) return;
    k_upsample<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, N, nx, Y, mean, stdv, U,
                                                          accumulate ? 1 : 0);
}

void launch_sub_f32(int64_t n, float* a, const float* b, cudaStream_t st) {
    if (n == 0) return;
    k_sub_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, b);
}

// Per-column mean and 1/std of targets [n][D].
__global__ void k_colstats(int64_t n, int D, const float* __restrict__ T, float* __restrict__ mean,
                           float* __restrict__ stdv, float* __restrict__ inv_std) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = 0; r < n; ++r) {
        const double v = T[r * D + c];
        s += v;
        s2 += v * v;
    }
    const double mu = s / n;
    double var = s2 / n - mu * mu;
    double sd = var > 0 ? sqrt(var) : 0.0;
    if (!(sd > 1e-30)) sd = 1.0;
    mean[c] = (float)mu;
    stdv[c] = (float)sd;
    inv_std[c] = (float)(1.0 / sd);
}

void launch_colstats(int64_t n, int D, const float* T, float* mean, float* stdv, float* inv_std,
                     cudaStream_t st) {
    k_colstats<<<(unsigned)((D + 127) / 128), 128, 0, st>>>(n, D, T, mean, stdv, inv_std);
}

__global__ void k_nonfinite_f32(int64_t n, const float* __restrict__ x, int* flag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t i = t; i < n; i += (int64_t)gridDim.x * blockDim.x) bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_nonfinite_f32(int64_t n, const float* x, int* flag, cudaStream_t st) {
    if (n == 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_nonfinite_f32<<<(unsigned)blocks, 256, 0, st>>>(n, x, flag);
}

}  // namespace klecgc
