// FP32 fine propagator, register-resident (with the CGC right-hand side;
// mixed modes).
//
// Each backward-Euler step of F is taken in increment form: with
// M = I + dt(A+cI), step m solves M delta_m = rhs_m and sets v += delta_m.
// The first right-hand side is rhs_1 = dt f0 - dt c v - dt A v (flux form);
// afterwards rhs_{m+1} = delta_m exactly, because M delta_m = rhs_m gives
// dt(A+cI) delta_m = rhs_m - delta_m, so dt f0 - dt(A+cI)(v + delta_m) =
// rhs_m - (rhs_m - delta_m) (the increments of backward Euler evolve by the
// source-free propagator, delta_{m+1} = M^{-1} delta_m), and such a step
// needs no operator application: a row costs its two LU recurrences, the
// carry correction and the accumulation of v.  Taken alone, though, this
// recurrence counts the rounding of delta_m again in every later increment
// (about J/2 times), where recomputing the right-hand side from v lets each
// rounding error decay like any state perturbation.  So the right-hand side
// is recomputed in flux form from v every kFluxEvery steps (and every step
// on the start values, in_mode 0, whose magnitude is that of the solution),
// which bounds the recount by kFluxEvery; on the increments of in_mode 1,
// whose size shrinks with the iteration, that keeps F0's rounding well below
// the solve's tolerance while 15 of 16 steps skip the operator.
// M is the same for every step, interval and iteration of a sample, so its
// LU factors are computed once per solve (FP64, rounded):
//     forward   y_i = rhs_i - l_i y_{i-1}
//     backward  x_i = dinv_i y_i - u_i x_{i+1}
// One warp owns QS systems (intervals n of one sample); lane k holds rows
// [kR, kR+R) of every system in registers for all J steps.  Both first-order
// recurrences are split at the lane boundaries: each lane runs its rows
// from a zero carry, the carries are propagated across the 32 lanes by a
// 5-level shuffle scan, and a correction adds carry * (product of the
// multipliers), y_i = yhat_i + F_i y_in, x_i = xhat_i + G_i x_in, where
//     F_j = prod_{k<=j} (-l_k),  G_j = prod_{k>=j} (-u_k)   (within the lane's rows)
// and the scan multipliers are products of whole-lane F/G: all of these are
// data independent and precomputed.  The coupled system is solved exactly
// (the same LU recurrences, regrouped); no reduced system is formed.
//
// Rows are padded to 32R >= nx + 1.  Padded rows have l = u = dinv = 0 so
// they stay 0 and act as the Dirichlet value beyond the last row; the table
// row nx still carries the weight of the boundary face nx (used by the
// flux-form first right-hand side).
//
// Output: the FP32 end values of every interval, fout[s][i][n].  F is affine,
// F(v + e) = F(v) + F0(e) with F0 the source-free propagator, so the caller
// runs F on the start values once (in_mode 0) and afterwards F0 on the FP32
// increments c = U^k - U^{k-1} (in_mode 1); the accumulation of F(U^k) in
// higher precision, the CGC right-hand side and the defect are formed by the
// CGC transform kernel that consumes fout.  The rounding of each F0 term is
// proportional to that term, so the iteration converges to its tolerance
// instead of stalling at FP32 resolution.
#include "common.cuh"

// Rounding does not depend on where the body is compiled: every product of
// the flux-form right-hand side is rounded on its own (__fmul_rn and friends
// are never fused into an FMA by the compiler), and every intended FMA is an
// explicit fmaf.  The same body runs in the per-solve kernel and in the
// persistent stage kernel of the uneven batch, whose results must agree bit
// for bit.

namespace klecgc {

constexpr int kFluxEvery = 16;

// Per-sample factor table, four arrays of [S][R][32] entries (row i = lane*R + j
// at index j*32 + lane):  GL = {G_j, l_j} for the ascending pass, FD =
// {F_j, dinv_j} and U = u_j for the descending pass, WD = wd_j = dt a_{i-1/2}/h^2
// for the first right-hand side.
struct Table32 {
    float2* GL;
    float2* FD;
    float* U;
    float* WD;
};

// One warp per sample; lane k owns rows [kR, kR + R).  The pivots of the LU
// factorization of M, piv_i = m_i - wl_i^2 / piv_{i-1} with m_i = 1 + wl_i +
// wr_i + dt c, form a continued fraction: (p_i, q_i) = (m_i p_{i-1} -
// wl_i^2 q_{i-1}, p_{i-1}) and piv_i = p_i / q_i.  Each lane multiplies the
// 2 x 2 maps of its rows (rescaled by powers of two, which is exact), an
// exclusive warp scan of these products gives every lane the pivot entering
// its first row, and each lane then runs the recurrence over its own rows
// in FP64 and writes their entries (consecutive lanes write consecutive
// words).  Padded rows (i >= nx) get l = u = dinv = 0.
__device__ __forceinline__ void mat2_rescale(double& a, double& b, double& c, double& d) {
    const double mx = fmax(fmax(fabs(a), fabs(b)), fmax(fabs(c), fabs(d)));
    if (mx > 0.0 && (mx > 0x1p+64 || mx < 0x1p-64)) {
        const int e = ilogb(mx);
        a = scalbn(a, -e);
        b = scalbn(b, -e);
        c = scalbn(c, -e);
        d = scalbn(d, -e);
    }
}

__global__ void __launch_bounds__(128) k_fine_table32(const double* __restrict__ a, int64_t S,
                                                      int nx, int R, double inv_h2, double dt,
                                                      double react, Table32 tb) {
    const int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= S) return;   // whole warps
    constexpr unsigned FULL = 0xffffffffu;
    const int Rt = 32 * R;
    const double* as = a + s * (nx + 1);
    float2* GL = tb.GL + s * (int64_t)Rt;
    float2* FD = tb.FD + s * (int64_t)Rt;
    float* Uu = tb.U + s * (int64_t)Rt;
    float* WD = tb.WD + s * (int64_t)Rt;
    const int i0 = lane * R;
    // product of this lane's maps, later rows on the left: T = M_{i0+R-1} ... M_{i0}
    double t00 = 1.0, t01 = 0.0, t10 = 0.0, t11 = 1.0;
    for (int j = 0; j < R; ++j) {
        const int i = i0 + j;
        if (i >= nx) break;
        const double wl = dt * as[i] * inv_h2, wr = dt * as[i + 1] * inv_h2;
        const double m = 1.0 + wl + wr + dt * react;
        const double c = i > 0 ? -wl * wl : 0.0;
        const double n00 = m * t00 + c * t10, n01 = m * t01 + c * t11;
        t10 = t00;
        t11 = t01;
        t00 = n00;
        t01 = n01;
        mat2_rescale(t00, t01, t10, t11);
    }
    // inclusive scan over lanes: X_k <- X_k X_{k-d}
    for (int d = 1; d < 32; d <<= 1) {
        const double b00 = __shfl_up_sync(FULL, t00, d), b01 = __shfl_up_sync(FULL, t01, d);
        const double b10 = __shfl_up_sync(FULL, t10, d), b11 = __shfl_up_sync(FULL, t11, d);
        if (lane >= d) {
            const double n00 = t00 * b00 + t01 * b10, n01 = t00 * b01 + t01 * b11;
            const double n10 = t10 * b00 + t11 * b10, n11 = t10 * b01 + t11 * b11;
            t00 = n00;
            t01 = n01;
            t10 = n10;
            t11 = n11;
            mat2_rescale(t00, t01, t10, t11);
        }
    }
    // exclusive prefix applied to (1, 0): the pivot before row i0 is p / q
    const double p = __shfl_up_sync(FULL, t00, 1), q = __shfl_up_sync(FULL, t10, 1);
    double piv = lane > 0 && q != 0.0 ? p / q : 1.0;
    for (int j = 0; j < R; ++j) {
        const int i = i0 + j;
        const int o = j * 32 + lane;
        const double wl = i <= nx ? dt * as[i] * inv_h2 : 0.0;
        double l = 0.0, dinv = 0.0, u = 0.0;
        if (i < nx) {
            const double wr = dt * as[i + 1] * inv_h2;
            double m = 1.0 + wl + wr + dt * react;
            if (i > 0) {
                l = -wl / piv;
                m -= wl * wl / piv;
            }
            piv = m;
            dinv = 1.0 / piv;
            u = (i + 1 < nx) ? -wr * dinv : 0.0;
        }
        GL[o] = make_float2(0.f, (float)l);
        WD[o] = (float)wl;
        FD[o] = make_float2(0.f, (float)dinv);
        Uu[o] = (float)u;
    }
    // within-lane products of the FP32-rounded multipliers (they must match
    // the local sweeps): F forward, G backward, formed in FP64
    double F = 1.0;
    for (int j = 0; j < R; ++j) {
        F *= -(double)GL[j * 32 + lane].y;
        FD[j * 32 + lane].x = (float)F;
    }
    double G = 1.0;
    for (int j = R - 1; j >= 0; --j) {
        G *= -(double)Uu[j * 32 + lane];
        GL[j * 32 + lane].x = (float)G;
    }
}

// The work of one CTA of 4 warps: intervals [part * 4 QS, part * 4 QS + 4 QS)
// of sample s, the sample's table staged in smem2 (R * 32 * 24 bytes).
template <int R, int QS, bool REACT>
__device__ __forceinline__ void fine32_cta(
    int64_t s, int part, int N, int nx, int J, float dt_react, float dt_f, int in_mode,
    const double* __restrict__ U64, const float2* __restrict__ Udf, const double* __restrict__ u0,
    const float* __restrict__ c32, Table32 tb, float* __restrict__ fout, float2* smem2) {
    float2* sGL = smem2;                 // [R][32] {G, l}
    float2* sFD = smem2 + R * 32;        // [R][32] {F, dinv}
    float* sU = reinterpret_cast<float*>(smem2 + 2 * R * 32);
    float* sWD = sU + R * 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = (part * (blockDim.x >> 5) + warp) * QS;
    {
        const int64_t off = s * (int64_t)(R * 32);
        for (int e = threadIdx.x; e < R * 32; e += blockDim.x) {
            sGL[e] = tb.GL[off + e];
            sFD[e] = tb.FD[off + e];
            sU[e] = tb.U[off + e];
            sWD[e] = tb.WD[off + e];
        }
    }
    __syncthreads();
    if (n0 >= N) return;
    constexpr unsigned FULL = 0xffffffffu;

    // data-independent scan multipliers
    float cf[5], cb[5];
    {
        float af = sFD[(R - 1) * 32 + lane].x;  // F_{R-1}: product over the lane's rows
        float ab = sGL[lane].x;                 // G_0
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int d = 1 << k;
            float pf = __shfl_up_sync(FULL, af, d);
            float pb = __shfl_down_sync(FULL, ab, d);
            cf[k] = lane >= d ? af : 0.f;
            cb[k] = lane + d <= 31 ? ab : 0.f;
            if (lane >= d) af *= pf;
            if (lane + d <= 31) ab *= pb;
        }
    }
    float gprev = __shfl_up_sync(FULL, sGL[(R - 1) * 32 + lane].x, 1);   // G_{R-1} of lane-1
    float wd_right = __shfl_down_sync(FULL, sWD[lane], 1);              // face right of row R-1
    if (lane == 0) gprev = 0.f;
    if (lane == 31) wd_right = 0.f;
    const int flux_every = in_mode == 0 ? 1 : kFluxEvery;
    const float src = in_mode == 0 ? dt_f : 0.f;

    float v[QS][R], w[QS][R];
    const int64_t sbase = s * (int64_t)nx * N;
#pragma unroll
    for (int q = 0; q < QS; ++q) {
        const int n = n0 + q;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int i = lane * R + j;
            float x0 = 0.f;
            if (i < nx && n < N) {
                const int64_t o = sbase + (int64_t)i * N + n - 1;
                if (in_mode == 1)
                    x0 = n > 0 ? c32[o] : 0.f;
                else if (n == 0)
                    x0 = (float)u0[i];
                else
                    x0 = Udf ? Udf[o].x : (float)U64[o];
            }
            v[q][j] = x0;
        }
    }
    // step-0 right-hand side and forward sweep (no pending update yet)
#pragma unroll
    for (int q = 0; q < QS; ++q) {
        float vl = __shfl_up_sync(FULL, v[q][R - 1], 1);
        float vr = __shfl_down_sync(FULL, v[q][0], 1);
        if (lane == 0) vl = 0.f;
        if (lane == 31) vr = 0.f;
        float fprev = __fmul_rn(sWD[lane], v[q][0] - vl);
        float yprev = 0.f;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const float lj = sGL[j * 32 + lane].y;
            const float wr = (j + 1 < R) ? sWD[(j + 1) * 32 + lane] : wd_right;
            const float vn = (j + 1 < R) ? v[q][j + 1] : vr;
            const float f = __fmul_rn(wr, vn - v[q][j]);
            float rhs = __fsub_rn(f, fprev);
            if (REACT) rhs = __fadd_rn(rhs, __fsub_rn(src, __fmul_rn(dt_react, v[q][j])));
            yprev = fmaf(-lj, yprev, rhs);
            w[q][j] = yprev;
            fprev = f;
        }
    }

    for (int step = 0; step < J; ++step) {
        // forward carries
        float yin[QS];
#pragma unroll
        for (int q = 0; q < QS; ++q) {
            float b = w[q][R - 1];
#pragma unroll
            for (int k = 0; k < 5; ++k) b = fmaf(cf[k], __shfl_up_sync(FULL, b, 1 << k), b);
            float t = __shfl_up_sync(FULL, b, 1);
            yin[q] = lane ? t : 0.f;
        }
        // descending: forward correction, diagonal, local backward sweep
        float xn[QS];
#pragma unroll
        for (int q = 0; q < QS; ++q) xn[q] = 0.f;
#pragma unroll
        for (int j = R - 1; j >= 0; --j) {
            const float2 fd = sFD[j * 32 + lane];
            const float uj = sU[j * 32 + lane];
#pragma unroll
            for (int q = 0; q < QS; ++q) {
                float y = fmaf(fd.x, yin[q], w[q][j]);
                float xh = fmaf(-uj, xn[q], __fmul_rn(y, fd.y));
                w[q][j] = xh;
                xn[q] = xh;
            }
        }
        // backward carries: z = true x at this lane's first row, zin = the
        // next lane's
        float z[QS], zin[QS];
#pragma unroll
        for (int q = 0; q < QS; ++q) {
            float b = w[q][0];
#pragma unroll
            for (int k = 0; k < 5; ++k) b = fmaf(cb[k], __shfl_down_sync(FULL, b, 1 << k), b);
            z[q] = b;
            float t = __shfl_down_sync(FULL, b, 1);
            zin[q] = lane < 31 ? t : 0.f;
        }
        const bool more = step + 1 < J;
        if (!more || (step + 1) % flux_every == 0) {
            // v += delta, then the next right-hand side in flux form from v
#pragma unroll
            for (int q = 0; q < QS; ++q) {
                // neighbour values after this step's update, for the next rhs
                float pl = __shfl_up_sync(FULL, v[q][R - 1] + w[q][R - 1], 1);
                float pr = __shfl_down_sync(FULL, v[q][0], 1);
                const float vl = lane ? fmaf(gprev, z[q], pl) : 0.f;
                const float vr = lane < 31 ? pr + zin[q] : 0.f;
                float fprev = 0.f, yprev = 0.f, lprev = 0.f;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const float2 gl = sGL[j * 32 + lane];
                    // The two rows next to a lane boundary must see bitwise-equal
                    // values there, or the flux through that face differs between
                    // them and the flux form stops being conservative.  The
                    // boundary rows are therefore updated by exactly the formulas
                    // the neighbouring lanes used for vl / vr above.
                    if (j == 0)
                        v[q][0] = v[q][0] + z[q];
                    else if (j == R - 1)
                        v[q][R - 1] = fmaf(gl.x, zin[q], v[q][R - 1] + w[q][R - 1]);
                    else
                        v[q][j] += fmaf(gl.x, zin[q], w[q][j]);
                    if (more) {
                        const float f = __fmul_rn(sWD[j * 32 + lane], v[q][j] - (j ? v[q][j - 1] : vl));
                        if (j) {
                            float rhs = __fsub_rn(f, fprev);
                            if (REACT) rhs = __fadd_rn(rhs, __fsub_rn(src, __fmul_rn(dt_react, v[q][j - 1])));
                            yprev = fmaf(-lprev, yprev, rhs);
                            w[q][j - 1] = yprev;
                        }
                        fprev = f;
                        lprev = gl.y;
                    }
                }
                if (more) {
                    const float f = __fmul_rn(wd_right, vr - v[q][R - 1]);
                    float rhs = __fsub_rn(f, fprev);
                    if (REACT) rhs = __fadd_rn(rhs, __fsub_rn(src, __fmul_rn(dt_react, v[q][R - 1])));
                    w[q][R - 1] = fmaf(-lprev, yprev, rhs);
                }
            }
        } else {
            // delta_j = xhat_j + G_j zin, v += delta, and the next step's
            // local forward sweep on the right-hand side delta
#pragma unroll
            for (int q = 0; q < QS; ++q) {
                float yprev = 0.f;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const float2 gl = sGL[j * 32 + lane];
                    const float d = fmaf(gl.x, zin[q], w[q][j]);
                    v[q][j] += d;
                    yprev = fmaf(-gl.y, yprev, d);
                    w[q][j] = yprev;
                }
            }
        }
    }

    // epilogue: F (in_mode 0) or F0(c) (in_mode 1) for this lane's rows, FP32
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = lane * R + j;
        if (i >= nx) break;
        float* o = fout + sbase + (int64_t)i * N + n0;
        if (QS == 2 && n0 + 1 < N) {
            *reinterpret_cast<float2*>(o) = make_float2(v[0][j], v[QS - 1][j]);
        } else {
#pragma unroll
            for (int q = 0; q < QS; ++q)
                if (n0 + q < N) o[q] = v[q][j];
        }
    }
}

template <int R, int QS, bool REACT>
__global__ void __launch_bounds__(128) k_fine32(
    int64_t S, int N, int nx, int J, int cps, float dt_react, float dt_f, int in_mode,
    const double* __restrict__ U64, const float2* __restrict__ Udf, const double* __restrict__ u0,
    const float* __restrict__ c32, Table32 tb, float* __restrict__ fout,
    const int* __restrict__ active) {
    extern __shared__ float2 smem2[];
    const int64_t s = blockIdx.x / cps;
    const int part = blockIdx.x - (int)(s * cps);
    if (!active[s]) return;
    fine32_cta<R, QS, REACT>(s, part, N, nx, J, dt_react, dt_f, in_mode, U64, Udf, u0, c32, tb,
                             fout, smem2);
}

int fine32_rows_per_lane(int nx) {
    const int need = (nx + 1 + 31) / 32;  // rows per lane so that 32R >= nx + 1
    for (int R : {2, 4, 8, 16, 32, 64})
        if (R >= need) return R;
    return 0;
}

size_t fine_table32_bytes(int64_t S, int R) { return (size_t)S * R * 32 * 24; }

void launch_fine_table32(const double* a, int64_t S, int nx, int R, double h, double dt,
                         double react, void* table, cudaStream_t st) {
    if (S == 0) return;
    const int64_t n = S * (int64_t)R * 32;
    char* p = static_cast<char*>(table);
    Table32 tb{reinterpret_cast<float2*>(p), reinterpret_cast<float2*>(p + 8 * n),
               reinterpret_cast<float*>(p + 16 * n), reinterpret_cast<float*>(p + 20 * n)};
    k_fine_table32<<<(unsigned)((S * 32 + 127) / 128), 128, 0, st>>>(a, S, nx, R, 1.0 / (h * h), dt,
                                                                      react, tb);
}

template <int R, int QS, bool REACT>
static void launch_r(int64_t S, int N, int nx, int J, double dt, double react, double forcing,
                     int in_mode, const double* U64, const float2* Udf, const double* u0,
                     const float* c32, const void* table, float* fout, const int* active,
                     cudaStream_t st) {
    constexpr int warps = 4;
    const int per_cta = warps * QS;
    const int cps = (N + per_cta - 1) / per_cta;
    const size_t smem = (size_t)R * 32 * 24;
    const int64_t n = S * (int64_t)R * 32;
    char* p = const_cast<char*>(static_cast<const char*>(table));
    Table32 tb{reinterpret_cast<float2*>(p), reinterpret_cast<float2*>(p + 8 * n),
               reinterpret_cast<float*>(p + 16 * n), reinterpret_cast<float*>(p + 20 * n)};
    static bool attr = false;
    if (!attr && smem > 48 * 1024) {
        cudaFuncSetAttribute(k_fine32<R, QS, REACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = true;
    }
    k_fine32<R, QS, REACT><<<(unsigned)(S * cps), warps * 32, smem, st>>>(
        S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0, c32,
        tb, fout, active);
}

template <int R, int QS>
static void launch_rr(int64_t S, int N, int nx, int J, double dt, double react, double forcing,
                      int in_mode, const double* U64, const float2* Udf, const double* u0,
                      const float* c32, const void* table, float* fout, const int* active,
                      cudaStream_t st) {
    const bool react_terms = react != 0.0 || (forcing != 0.0 && in_mode == 0);
    if (react_terms)
        launch_r<R, QS, true>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table,
                              fout, active, st);
    else
        launch_r<R, QS, false>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table,
                               fout, active, st);
}

void launch_fine32(int64_t S, int N, int nx, int J, double dt, double react, double forcing,
                   int in_mode, const double* U64, const float2* Udf, const double* u0,
                   const float* c32, const void* table, float* fout, const int* active,
                   cudaStream_t st) {
    if (S == 0) return;
    switch (fine32_rows_per_lane(nx)) {
#define KLECGC_F32(RR, QQ)                                                                   \
    case RR:                                                                                 \
        launch_rr<RR, QQ>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table, \
                          fout, active, st);                                                  \
        break;
        KLECGC_F32(2, 2)
        KLECGC_F32(4, 2)
        KLECGC_F32(8, 2)
        KLECGC_F32(16, 2)
        KLECGC_F32(32, 2)
        KLECGC_F32(64, 1)
#undef KLECGC_F32
        default: break;
    }
}

}  // namespace klecgc

// ---- the uneven batch: the fine stage as one persistent launch
namespace klecgc {

// Intervals per CTA task: 4 warps x QS systems (QS = 1 at 64 rows per lane,
// for registers, else 2).
static __host__ __device__ int fine32_qs(int R) { return R >= 64 ? 1 : 2; }

int batch_fine_parts(int N, int R) {
    const int per = 4 * fine32_qs(R);
    return (N + per - 1) / per;
}

size_t batch_fine_smem(int R) { return (size_t)R * 32 * 24; }

__device__ __forceinline__ int batch_next_fine(int* queue, int* s_task) {
    if (threadIdx.x == 0) *s_task = atomicAdd(queue, 1);
    __syncthreads();
    const int t = *s_task;
    __syncthreads();
    return t;
}

// One launch per (R, reaction terms) group of classes: the body is compiled
// for one row count, so its registers are those of the standalone kernel
// (one kernel over every R spilled).  REACT = true is exact also without the
// terms (it adds dt f0 - dt c v = 0 exactly), so a class with forcing uses it
// in every iteration.
template <int R, bool REACT>
__global__ void __launch_bounds__(128) k_batch_fine(const BatchClass* __restrict__ cls,
                                                    const BatchTask* __restrict__ tasks,
                                                    int ntasks, int* queue, int k_host,
                                                    const int* __restrict__ kdev) {
    constexpr int QS = R >= 64 ? 1 : 2;
    extern __shared__ float2 smem2[];
    __shared__ int s_task;
    const int k = kdev ? *kdev : k_host;
    const int in_mode = k == 0 ? 0 : 1;
    for (;;) {
        const int t = batch_next_fine(queue, &s_task);
        if (t >= ntasks) break;
        const BatchTask tk = tasks[t];
        const BatchClass& C = cls[tk.c];
        if (!C.active[tk.s]) continue;
        const int64_t n = C.S * (int64_t)R * 32;
        const char* p = C.tab32;
        Table32 tb{reinterpret_cast<float2*>(const_cast<char*>(p)),
                   reinterpret_cast<float2*>(const_cast<char*>(p + 8 * n)),
                   reinterpret_cast<float*>(const_cast<char*>(p + 16 * n)),
                   reinterpret_cast<float*>(const_cast<char*>(p + 20 * n))};
        fine32_cta<R, QS, REACT>(tk.s, tk.part, C.N, C.nx, C.J, C.dt_react, C.dt_f, in_mode,
                                 C.defect ? nullptr : C.U, C.defect ? C.Udf : nullptr, C.u0,
                                 C.c32, tb, C.fout, smem2);
        __syncthreads();
    }
}

template <int R, bool REACT>
static void batch_fine_rr(const BatchClass* cls, const BatchTask* tasks, int ntasks, int* queue,
                          int k_host, const int* kdev, int grid, cudaStream_t st) {
    const size_t smem = batch_fine_smem(R);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_batch_fine<R, REACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = true;
    }
    if (grid <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_fine<R, REACT>, 128,
                                                          smem) != cudaSuccess || per < 1)
            per = 1;
        grid = sms * per;
    }
    k_batch_fine<R, REACT><<<grid, 128, smem, st>>>(cls, tasks, ntasks, queue, k_host, kdev);
}

void launch_batch_fine(const BatchClass* cls, const BatchTask* tasks, int ntasks, int* queue,
                       int k_host, const int* kdev, int R, int rt, int grid, cudaStream_t st) {
    if (ntasks == 0) return;
#define KLECGC_BFR(RR)                                                                         \
    case RR:                                                                                   \
        if (rt)                                                                                \
            batch_fine_rr<RR, true>(cls, tasks, ntasks, queue, k_host, kdev, grid, st);       \
        else                                                                                   \
            batch_fine_rr<RR, false>(cls, tasks, ntasks, queue, k_host, kdev, grid, st);      \
        break;
    switch (R) {
        KLECGC_BFR(2)
        KLECGC_BFR(4)
        KLECGC_BFR(8)
        KLECGC_BFR(16)
        KLECGC_BFR(32)
        KLECGC_BFR(64)
        default: break;
    }
#undef KLECGC_BFR
}

}  // namespace klecgc
