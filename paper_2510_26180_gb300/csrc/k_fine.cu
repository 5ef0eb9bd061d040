// Fine propagator F and the CGC right-hand side.
//
// Step 1 of Algorithm 2 (eq. PGC_step1): on every subinterval n, J backward-
// Euler steps (I + dt(A + cI)) v' = v + dt f0 from start_1 = u0 and
// start_n = U^k_{n-1}.  The epilogue forms the CGC right-hand side of
// eq. matrix_NT at the Newton point of eq. Newton2,
//     r_n = (I + dT(A + cI)) F_n - prev_n,  prev_1 = alpha U_N, prev_n = U_{n-1},
// which equals (I + dT(A+cI)) b_n + dT f0 for the jump b_n of Section 3.2
// (the coarse solves G(.) in b_n cancel against (I + dT(A+cI))).
//
// Internal layout: U, r are [S][nx][N] (time fastest).  Thread (s, n) owns
// column n of sample s; a warp touches 32 consecutive n of one row, so every
// state access is a coalesced 128/256-byte transaction.
#include "common.cuh"

namespace klecgc {

__device__ __forceinline__ double prev_value(const double* Us, int i, int n, int N, double alpha) {
    return n == 0 ? alpha * Us[(int64_t)i * N + (N - 1)] : Us[(int64_t)i * N + (n - 1)];
}

// FP64: direct Thomas on the LU factors of M_F, state in place in r.
// jump = 0 leaves the fine end values F_n themselves in r (classical parareal).
__global__ void __launch_bounds__(128) k_fine_sweep_fp64(
    int64_t S, int N, int nx, int J, double dT, double alpha, double dTreact, double dtf,
    const double* __restrict__ U, const double* __restrict__ u0, const FineCoef64* __restrict__ fc,
    const double* __restrict__ wT, double* __restrict__ r, const int* __restrict__ active,
    int jump) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t s = t / N;
    int n = (int)(t - s * N);
    if (s >= S || !active[s]) return;
    const int64_t base = s * (int64_t)nx * N;
    const double* Us = U + base;
    double* rs = r + base;
    const FineCoef64* c = fc + s * (nx + 1);
    for (int i = 0; i < nx; ++i) rs[(int64_t)i * N + n] = n == 0 ? u0[i] : Us[(int64_t)i * N + n - 1];
    for (int j = 0; j < J; ++j) {
        double y = 0.0;
        for (int i = 0; i < nx; ++i) {
            double* p = rs + (int64_t)i * N + n;
            y = fma(-c[i].l, y, *p + dtf);
            *p = y;
        }
        double x = 0.0;
        for (int i = nx - 1; i >= 0; --i) {
            double* p = rs + (int64_t)i * N + n;
            x = fma(c[i + 1].wd, x, *p) * c[i].dinv;
            *p = x;
        }
    }
    if (!jump) return;
    // the jump reads F at rows i-1..i+1 of its own column: write r into the
    // same column only after F_{i+1} has been read (sliding window below).
    double Fm = 0.0, Fi = rs[n];
    const double* wTs = wT + s * (nx + 1);
    for (int i = 0; i < nx; ++i) {
        double Fp = (i + 1 < nx) ? rs[(int64_t)(i + 1) * N + n] : 0.0;
        double BF = Fi + wTs[i] * (Fi - Fm) - wTs[i + 1] * (Fp - Fi) + dTreact * Fi;
        rs[(int64_t)i * N + n] = BF - prev_value(Us, i, n, N, alpha);
        Fm = Fi;
        Fi = Fp;
    }
}

void launch_fine_sweep_fp64(int64_t S, int N, int nx, int J, double dT, double alpha, double react,
                            double forcing, const double* U, const double* u0,
                            const FineCoef64* fc, const double* wT, double* r, const int* active,
                            cudaStream_t st, int jump) {
    int64_t n = S * N;
    if (n == 0) return;
    double dt = dT / J;
    k_fine_sweep_fp64<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
        S, N, nx, J, dT, alpha, dT * react, dt * forcing, U, u0, fc, wT, r, active, jump);
}

// Sequential correction of classical parareal (Algorithm 1, eq. pred_correc):
//     U^{k+1}_n = G(U^{k+1}_{n-1}) + F(U^k_{n-1}) - G(U^k_{n-1}),  U_0 = u0,
// G one backward-Euler step of dT (LU factors gc of I + dT(A + cI)).  One
// thread per sample; F: the fine end values [S][nx][N]; U is updated in place
// (G(U^k_{n-1}) is taken before U_{n-1} is overwritten); scratch [2][nx][S]
// holds G(U^k_{n-1}) and the new start value.  delta[s] receives the bit
// pattern of max_n ||U^{k+1}_n - U^k_n||_inf (NaN kept).
__device__ __forceinline__ void be_solve_col(const FineCoef64* c, int nx, double dtf, double* v,
                                             int64_t stride) {
    double y = 0.0;
    for (int i = 0; i < nx; ++i) {
        y = fma(-c[i].l, y, v[i * stride] + dtf);
        v[i * stride] = y;
    }
    double x = 0.0;
    for (int i = nx - 1; i >= 0; --i) {
        x = fma(c[i + 1].wd, x, v[i * stride]) * c[i].dinv;
        v[i * stride] = x;
    }
}

__global__ void __launch_bounds__(64) k_parareal_correct(
    int64_t S, int N, int nx, double dTf, const double* __restrict__ u0,
    const FineCoef64* __restrict__ gc, const double* __restrict__ F, double* __restrict__ U,
    double* __restrict__ scratch, unsigned long long* __restrict__ delta,
    const int* __restrict__ active) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S || !active[s]) return;
    const FineCoef64* c = gc + s * (nx + 1);
    double* gold = scratch + s;                  // [nx][S]
    double* vnew = scratch + (int64_t)nx * S + s;
    const double* Fs = F + s * (int64_t)nx * N;
    double* Us = U + s * (int64_t)nx * N;
    // G(U^k_0 := u0) and the new start value u0
    for (int i = 0; i < nx; ++i) {
        gold[(int64_t)i * S] = u0[i];
        vnew[(int64_t)i * S] = u0[i];
    }
    be_solve_col(c, nx, dTf, gold, S);
    double dmax = 0.0;
    bool bad = false;
    for (int n = 0; n < N; ++n) {
        be_solve_col(c, nx, dTf, vnew, S);   // G(U^{k+1}_{n-1})
        for (int i = 0; i < nx; ++i) {
            const int64_t o = (int64_t)i * N + n;
            const double uold = Us[o];
            const double unew = vnew[(int64_t)i * S] + Fs[o] - gold[(int64_t)i * S];
            gold[(int64_t)i * S] = uold;     // start of G(U^k_n) for the next n
            vnew[(int64_t)i * S] = unew;
            Us[o] = unew;
            const double d = fabs(unew - uold);
            dmax = fmax(dmax, d);
            bad |= d != d;
        }
        if (n + 1 < N) be_solve_col(c, nx, dTf, gold, S);  // G(U^k_n)
    }
    delta[s] = bad ? 0x7ff8000000000000ull : (unsigned long long)__double_as_longlong(dmax);
}

void launch_parareal_correct(int64_t S, int N, int nx, double dTf, const double* u0,
                             const FineCoef64* gc, const double* F, double* U, double* scratch,
                             unsigned long long* delta, const int* active, cudaStream_t st) {
    if (S == 0) return;
    k_parareal_correct<<<(unsigned)((S + 63) / 64), 64, 0, st>>>(S, N, nx, dTf, u0, gc, F, U,
                                                                scratch, delta, active);
}

// r = (I + dT(A + cI)) F - prev in FP64 for an FP32 F (stage entry of the
// mixed fine sweep): one thread per (sample, interval), rows in sequence.
__global__ void k_jump_from_f32(int64_t S, int N, int nx, double alpha, double dTreact,
                                const float* __restrict__ F, const double* __restrict__ U,
                                const double* __restrict__ wT, double* __restrict__ r) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t s = t / N;
    int n = (int)(t - s * N);
    if (s >= S) return;
    const int64_t base = s * (int64_t)nx * N;
    const double* wTs = wT + s * (nx + 1);
    double Fm = 0.0, Fi = F[base + n];
    for (int i = 0; i < nx; ++i) {
        const double Fp = (i + 1 < nx) ? (double)F[base + (int64_t)(i + 1) * N + n] : 0.0;
        const double BF = Fi + wTs[i] * (Fi - Fm) - wTs[i + 1] * (Fp - Fi) + dTreact * Fi;
        r[base + (int64_t)i * N + n] = BF - prev_value(U + base, i, n, N, alpha);
        Fm = Fi;
        Fi = Fp;
    }
}

void launch_jump_from_f32(int64_t S, int N, int nx, double alpha, double dTreact, const float* F,
                          const double* U, const double* wT, double* r, cudaStream_t st) {
    int64_t n = S * N;
    if (n == 0) return;
    k_jump_from_f32<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(S, N, nx, alpha, dTreact, F, U,
                                                                 wT, r);
}

// Reference solution U*: N*J sequential backward-Euler steps per sample, one
// thread per sample, state in scratch[nx][S] (samples interleaved so that a
// warp's accesses coalesce).  Output U[s][i][n] (internal layout).
__global__ void __launch_bounds__(64) k_fine_sequential(int64_t S, int N, int nx, int J,
                                                        double dtf, const double* __restrict__ u0,
                                                        const FineCoef64* __restrict__ fc,
                                                        double* __restrict__ scratch,
                                                        double* __restrict__ U) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S) return;
    const FineCoef64* c = fc + s * (nx + 1);
    for (int i = 0; i < nx; ++i) scratch[(int64_t)i * S + s] = u0[i];
    double* Us = U + s * (int64_t)nx * N;
    for (int n = 0; n < N; ++n) {
        for (int j = 0; j < J; ++j) {
            double y = 0.0;
            for (int i = 0; i < nx; ++i) {
                double* p = scratch + (int64_t)i * S + s;
                y = fma(-c[i].l, y, *p + dtf);
                *p = y;
            }
            double x = 0.0;
            for (int i = nx - 1; i >= 0; --i) {
                double* p = scratch + (int64_t)i * S + s;
                x = fma(c[i + 1].wd, x, *p) * c[i].dinv;
                *p = x;
            }
        }
        for (int i = 0; i < nx; ++i) Us[(int64_t)i * N + n] = scratch[(int64_t)i * S + s];
    }
}

void launch_fine_sequential(int64_t S, int N, int nx, int J, double dt_forcing, const double* u0,
                            const FineCoef64* fc, double* scratch, double* U, cudaStream_t st) {
    if (S == 0) return;
    k_fine_sequential<<<(unsigned)((S + 63) / 64), 64, 0, st>>>(S, N, nx, J, dt_forcing, u0, fc,
                                                                scratch, U);
}

}  // namespace klecgc
