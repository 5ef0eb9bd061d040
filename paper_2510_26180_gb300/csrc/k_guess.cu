// Surrogate guess (gPC basis and contraction) and the dense products of the setup.
//
//  psi_j(xi) = prod_l psi_{k_l}(xi_l), |k|_1 <= p              (Section 2.2, eq. complete)
//  U^0(xi)   = ubar + sum_k sqrt(lambda_k) (sum_j h_kj psi_j(xi)) g_k
//            = ubar + psi(xi) W,   W = H diag(sqrt(lambda)) G   (Algorithm 3, step 6)
#include "common.cuh"

namespace klecgc {

// Orthonormal Hermite values by psi_{m+1} = (x psi_m - sqrt(m) psi_{m-1}) / sqrt(m+1).
__device__ __forceinline__ double hermite_on(int k, double x) {
    double pm = 1.0, pc = x;
    if (k == 0) return 1.0;
    for (int m = 1; m < k; ++m) {
        double pn = (x * pc - sqrt((double)m) * pm) / sqrt((double)(m + 1));
        pm = pc;
        pc = pn;
    }
    return pc;
}

// psi[s][j] for j < P; row stride ld >= P, columns P..ld-1 set to 0.
template <typename T>
__global__ void k_psi(const double* __restrict__ xi, int64_t S, int M,
                      const int* __restrict__ degrees, int P, int ld, T* __restrict__ psi) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * ld) return;
    int64_t s = t / ld;
    int j = (int)(t - s * ld);
    if (j >= P) {
        psi[t] = (T)0;
        return;
    }
    double v = 1.0;
    for (int l = 0; l < M; ++l) {
        int k = degrees[j * M + l];
        if (k) v *= hermite_on(k, xi[s * M + l]);
    }
    psi[t] = (T)v;
}

template <typename T>
void launch_psi(const double* xi, int64_t S, int M, const int* degrees, int P, T* psi, int ld,
                cudaStream_t st) {
    int64_t n = S * ld;
    if (n == 0) return;
    k_psi<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xi, S, M, degrees, P, ld, psi);
}
template void launch_psi<double>(const double*, int64_t, int, const int*, int, double*, int,
                                 cudaStream_t);
template void launch_psi<float>(const double*, int64_t, int, const int*, int, float*, int,
                                cudaStream_t);

// Tiled SIMT product, 64x64 output tile, 16-deep k slices, 4x4 outputs per thread.
// Accumulates in T; the FP64 column bias and the previous C are added in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(int64_t Mr, int64_t Nc, int64_t K, const T* A,
                                              int64_t lda_m, int64_t lda_k, const T* B,
                                              int64_t ldb_k, int64_t ldb_n, double* C,
                                              int64_t ldc, bool accumulate,
                                              const double* col_bias) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = blockIdx.y * (int64_t)BM, n0 = blockIdx.x * (int64_t)BN;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BK * BM; e += 256) {
            int kk = e / BM, mm = e % BM;
            int64_t gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < Mr && gk < K) ? A[gm * lda_m + gk * lda_k] : (T)0;
        }
        for (int e = tid; e < BK * BN; e += 256) {
            int kk = e / BN, nn = e % BN;
            int64_t gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < Nc && gk < K) ? B[gk * ldb_k + gn * ldb_n] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t gm = m0 + ty + 16 * i;
        if (gm >= Mr) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gn = n0 + tx + 16 * j;
            if (gn >= Nc) continue;
            double v = (double)acc[i][j];
            if (col_bias) v += col_bias[gn];
            double* c = C + gm * ldc + gn;
            *c = accumulate ? *c + v : v;
        }
    }
}

template <typename T>
void launch_gemm(int64_t Mr, int64_t Nc, int64_t K, const T* A, int64_t lda_m, int64_t lda_k,
                 const T* B, int64_t ldb_k, int64_t ldb_n, double* C, int64_t ldc, bool accumulate,
                 const double* col_bias, cudaStream_t st) {
    if (Mr == 0 || Nc == 0) return;
    dim3 grid((unsigned)((Nc + 63) / 64), (unsigned)((Mr + 63) / 64));
    k_gemm<T><<<grid, 256, 0, st>>>(Mr, Nc, K, A, lda_m, lda_k, B, ldb_k, ldb_n, C, ldc,
                                     accumulate, col_bias);
}
template void launch_gemm<double>(int64_t, int64_t, int64_t, const double*, int64_t, int64_t,
                                  const double*, int64_t, int64_t, double*, int64_t, bool,
                                  const double*, cudaStream_t);
template void launch_gemm<float>(int64_t, int64_t, int64_t, const float*, int64_t, int64_t,
                                 const float*, int64_t, int64_t, double*, int64_t, bool,
                                 const double*, cudaStream_t);

// Column means of Y[rows][cols] into mean[cols], then Y -= mean (row-wise).
__global__ void k_mean_center(double* Y, int64_t rows, int64_t cols, double* mean) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double acc = 0.0;
    for (int64_t r = 0; r < rows; ++r) acc += Y[r * cols + c];
    double m = acc / (double)rows;
    mean[c] = m;
    for (int64_t r = 0; r < rows; ++r) Y[r * cols + c] -= m;
}

void launch_mean_center(double* Y, int64_t rows, int64_t cols, double* mean, cudaStream_t st) {
    if (cols == 0) return;
    k_mean_center<<<(unsigned)((cols + 255) / 256), 256, 0, st>>>(Y, rows, cols, mean);
}

__global__ void k_to_float(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) y[t] = (float)x[t];
}

void launch_to_float(const double* x, float* y, int64_t n, cudaStream_t st) {
    if (n == 0) return;
    k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
}

}  // namespace klecgc
