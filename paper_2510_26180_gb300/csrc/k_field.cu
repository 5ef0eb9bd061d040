// Coefficient field and per-sample factorizations.
//
//  a(x_{i+1/2}; xi) = exp(sum_m sqrt(lambda_m) phi_m(x_{i+1/2}) xi_m)  (input KL)
//  M_F = I + dt (A + c I)                     fine backward-Euler matrix (Section 3.1)
//  M_k = lambda_k I + dT (A + c I)            shifted CGC systems, eq. three steps (b)
// A is the 3-point flux-form operator with face coefficients a/h^2.  The
// factorizations are computed once per solve and reused by every iteration.
#include "common.cuh"

namespace klecgc {

__global__ void k_field(const double* __restrict__ xi, int64_t S, int M,
                        const double* __restrict__ basis, int nf, double* __restrict__ a) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * nf) return;
    int64_t s = t / nf;
    int f = (int)(t - s * nf);
    double g = 0.0;
    for (int m = 0; m < M; ++m) g = fma(basis[(int64_t)m * nf + f], xi[s * M + m], g);
    a[t] = exp(g);
}

void launch_field(const double* xi, int64_t S, int M, const double* basis, int nf, double* a,
                  cudaStream_t st) {
    int64_t n = S * nf;
    if (n == 0) return;
    k_field<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xi, S, M, basis, nf, a);
}

__global__ void k_face_weights(const double* __restrict__ a, int64_t n, double scale,
                               double* __restrict__ w) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) w[t] = scale * a[t];
}

void launch_face_weights(const double* a, int64_t S, int nf, double scale, double* w,
                         cudaStream_t st) {
    int64_t n = S * nf;
    if (n == 0) return;
    k_face_weights<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, n, scale, w);
}

// One thread per sample: LU of the symmetric tridiagonal M_F.  Row i couples
// to row i-1 through face i: M_{i,i-1} = M_{i-1,i} = -wd_i, wd_f = dt a_f / h^2.
// Entry nx of each sample holds only wd_nx (the right boundary face).
// The pivots are formed without cancellation: with lambda' = 1 + dt c,
//     piv_i = wd_{i+1} + sigma_i,  sigma_0 = lambda' + wd_0,
//     sigma_i = lambda' + wd_i sigma_{i-1} / piv_{i-1}  (piv_{i-1} = wd_i + sigma_{i-1}),
// which equals piv_i = M_ii - wd_i^2 / piv_{i-1} in exact arithmetic but never
// subtracts O(wd) numbers: the small part sigma, which carries the smooth
// modes, keeps full relative precision however large dt a / h^2 is.
__global__ void k_fine_factors(const double* __restrict__ a, int64_t S, int nx, double inv_h2,
                               double dt, double react, FineCoef64* __restrict__ f64,
                               FineCoef32* __restrict__ f32) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double* as = a + s * (nx + 1);
    FineCoef64* o64 = f64 + s * (nx + 1);
    FineCoef32* o32 = f32 ? f32 + s * (nx + 1) : nullptr;
    const double lam = 1.0 + dt * react;
    double wl = dt * as[0] * inv_h2;
    double sig = lam + wl, piv = 1.0;
    for (int i = 0; i < nx; ++i) {
        const double wr = dt * as[i + 1] * inv_h2;
        double l = 0.0;
        if (i > 0) {
            l = -wl / piv;           // M_{i,i-1} / piv_{i-1}
            sig = lam - l * sig;     // lambda' + wl sigma_{i-1} / piv_{i-1}
        }
        piv = wr + sig;
        const double dinv = 1.0 / piv;
        o64[i] = FineCoef64{l, dinv, wl, 0.0};
        if (o32) o32[i] = FineCoef32{(float)l, (float)dinv, (float)wl, 0.0f};
        wl = wr;
    }
    o64[nx] = FineCoef64{0.0, 0.0, wl, 0.0};
    if (o32) o32[nx] = FineCoef32{0.0f, 0.0f, (float)wl, 0.0f};
}

void launch_fine_factors(const double* a, int64_t S, int nx, double h, double dt, double react,
                         FineCoef64* f64, FineCoef32* f32, cudaStream_t st) {
    if (S == 0) return;
    k_fine_factors<<<(unsigned)((S + 127) / 128), 128, 0, st>>>(a, S, nx, 1.0 / (h * h), dt,
                                                                 react, f64, f32);
}

// One thread per (sample, frequency k): LDU of M_k with complex diagonal
// lambda_k + dT(w_i + w_{i+1} + c) and real off-diagonal -dT w_i.  Stored
// per (s, i, k): dinv_i = 1/piv_i and lu_i = M_{i,i+1} dinv_i, layout
// [S][nx][K] so that the K systems of one sample are contiguous per row.
// ext (optional, [S][nx]): a per-row addition dT ext_i to the diagonal (the
// averaged Jacobian of the nonlinear CGC).
// Pivots without cancellation (lambda'_i = lambda_k + dT c + dT ext_i,
// W_i = dT w_i):  piv_i = W_{i+1} + sigma_i,  sigma_0 = lambda'_0 + W_0,
//     sigma_i = lambda'_i + W_i sigma_{i-1} / piv_{i-1}.
// The textbook form piv_i = delta_i - W_i^2 / piv_{i-1} subtracts numbers of
// size W (~1e4 at nx = 1023, dT = 1/64) to leave sigma (~|lambda_k|^{1/2} W^{1/2}):
// in FP64 that kept ~1e-11 of the smooth modes, and step (c) multiplies the
// loss by up to alpha^{-(N-1)/N} (1e4 at alpha = 1e-4, N = 64): a 2e-9
// relative error of one CGC application there; this form leaves 6e-12.
template <typename T>
__global__ void k_cgc_factors(const double* __restrict__ a, int64_t S, int nx, double wscale,
                              double dTreact, const double2* __restrict__ lam, int K,
                              Cplx<T>* __restrict__ dinv, Cplx<T>* __restrict__ lu,
                              const double* __restrict__ ext, double dT) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * K) return;
    int64_t s = t / K;
    int k = (int)(t - s * K);
    const double* as = a + s * (nx + 1);
    const double2 lk = lam[k];
    double wl = wscale * as[0];
    double sr = 0.0, si = 0.0;   // sigma_{i-1}
    double ir = 0.0, ii = 0.0;   // 1 / piv_{i-1}
    for (int i = 0; i < nx; ++i) {
        const double wr = wscale * as[i + 1];
        double lr = lk.x + dTreact, li = lk.y;
        if (ext) lr += dT * ext[s * nx + i];
        if (i == 0) {
            sr = lr + wl;
            si = li;
        } else {
            // sigma_i = lambda'_i + wl * sigma_{i-1} / piv_{i-1}
            const double qr = sr * ir - si * ii, qi = sr * ii + si * ir;
            sr = lr + wl * qr;
            si = li + wl * qi;
        }
        const double pr = wr + sr, pi = si;  // piv_i
        const double inv = 1.0 / (pr * pr + pi * pi);
        ir = pr * inv;
        ii = -pi * inv;
        int64_t o = (s * nx + i) * K + k;
        dinv[o] = Cplx<T>{(T)ir, (T)ii};
        double ur = (i + 1 < nx) ? -wr * ir : 0.0, ui = (i + 1 < nx) ? -wr * ii : 0.0;
        lu[o] = Cplx<T>{(T)ur, (T)ui};
        wl = wr;
    }
}

template <typename T>
void launch_cgc_factors(const double* a, int64_t S, int nx, double h, double dT, double react,
                        const double2* lam, int K, Cplx<T>* dinv, Cplx<T>* lu, cudaStream_t st,
                        const double* ext) {
    int64_t n = S * K;
    if (n == 0) return;
    k_cgc_factors<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
        a, S, nx, dT / (h * h), dT * react, lam, K, dinv, lu, ext, dT);
}
template void launch_cgc_factors<double>(const double*, int64_t, int, double, double, double,
                                         const double2*, int, Cplx<double>*, Cplx<double>*,
                                         cudaStream_t, const double*);
template void launch_cgc_factors<float>(const double*, int64_t, int, double, double, double,
                                        const double2*, int, Cplx<float>*, Cplx<float>*,
                                        cudaStream_t, const double*);

// FP32 variant for the defect path, whose CGC is an FP32 approximate inverse.
// With lambda' = lambda_k + dT c and w_i = dT a_{i-1/2}/h^2, the pivots are
// written piv_i = w_{i+1} + sigma_i with
//     sigma_0 = lambda' + w_0,  sigma_i = lambda' + w_i sigma_{i-1} / (w_i + sigma_{i-1}),
// which is the same recurrence as piv_i = delta_i - w_i^2/piv_{i-1} but free of
// cancellation: the small part sigma, which carries the smooth modes, never
// emerges from differences of O(w) numbers, so FP32 keeps it accurate.
__global__ void k_cgc_factors32(const float* __restrict__ wT32, int64_t S, int nx, float dTreact,
                                const float2* __restrict__ lam, int K,
                                Cplx<float>* __restrict__ dinv, Cplx<float>* __restrict__ lu) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * K) return;
    int64_t s = t / K;
    int k = (int)(t - s * K);
    const float* ws = wT32 + s * (nx + 1);
    const float2 lk = lam[k];
    const float lr = lk.x + dTreact, li = lk.y;
    float sr = lr + ws[0], si = li;  // sigma_0
    for (int i = 0; i < nx; ++i) {
        const float wr = ws[i + 1];
        if (i > 0) {
            // sigma_i = lambda' + w_i sigma / (w_i + sigma)
            const float wl = ws[i];
            const float br = wl + sr, bi = si;
            const float inv = 1.f / (br * br + bi * bi);
            const float qr = (sr * br + si * bi) * inv, qi = (si * br - sr * bi) * inv;
            sr = lr + wl * qr;
            si = li + wl * qi;
        }
        const float pr = wr + sr, pi = si;  // piv_i = w_{i+1} + sigma_i
        const float den = pr * pr + pi * pi;
        const float ir = pr / den, ii = -pi / den;
        const int64_t o = (s * nx + i) * K + k;
        dinv[o] = Cplx<float>{ir, ii};
        lu[o] = (i + 1 < nx) ? Cplx<float>{-wr * ir, -wr * ii} : Cplx<float>{0.f, 0.f};
    }
}

void launch_cgc_factors32(const float* wT32, int64_t S, int nx, double dTreact,
                          const float2* lam, int K, Cplx<float>* dinv, Cplx<float>* lu,
                          cudaStream_t st) {
    int64_t n = S * K;
    if (n == 0) return;
    k_cgc_factors32<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(wT32, S, nx, (float)dTreact, lam,
                                                                  K, dinv, lu);
}

__global__ void k_nonfinite(const double* __restrict__ x, int64_t n, int* flag) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t i = t; i < n; i += (int64_t)gridDim.x * blockDim.x) bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_nonfinite_flag(const double* x, int64_t n, int* flag, cudaStream_t st) {
    if (n == 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_nonfinite<<<(unsigned)blocks, 256, 0, st>>>(x, n, flag);
}

}  // namespace klecgc
