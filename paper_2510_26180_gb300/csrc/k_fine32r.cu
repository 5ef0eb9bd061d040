// FP32 fine propagator, one interval per warp with every LU factor in
// registers (mixed modes).
//
// The same computation as k_fine32 (J backward-Euler steps of
// M = I + dt(A + cI) per interval in increment form, the right-hand side in
// flux form from v every kFluxEvery32r steps and in every step on start
// values), with the rows of one interval split over the 32 lanes of a warp
// (lane g owns rows [g R, g R + R)).  A warp holds the factors of its lane's
// rows in registers (5 R floats) and runs L intervals of its sample one after
// another, so the factors are read once per L intervals and the inner loop
// touches no shared memory.
//
// Per step the partitioned LU solve is regrouped so that neither carry scan
// stalls the local sweeps.  With yhat the local forward sweep of the
// right-hand side (zero carry into the lane) and
//     F_j = prod_{k<=j} (-l_k),   G_j = prod_{k>=j} (-u_k)
// the true forward values are y = yhat + F yin and the true solution is
// x = xhat(y) + G zin, xhat the local backward sweep (zero carry from the
// right).  xhat is linear, so
//     x_j = X_j + yin P_j + zin G_j,   X = xhat(yhat),   P = xhat(F),
// where P_j = dinv_j F_j - u_j P_{j+1} (P_R = 0) is data independent.  The
// next step's right-hand side is x itself (increment form), and its local
// forward sweep is linear too: fwd(x) = fwd(e) + zin Hg with e = X + yin P
// and Hg = fwd(G) (Hg_j = G_j - l_j Hg_{j-1}), again data independent.  A
// step is then
//   1. the forward carry scan over the lanes' yhat_{R-1} (multiplier F_{R-1}),
//      interleaved with the backward sweep X_j = dinv_j yhat_j - u_j X_{j+1};
//   2. the backward carry scan over x at each lane's first row,
//      X_0 + yin P_0 (multiplier G_0), interleaved with e_j = X_j + yin P_j,
//      v_j += e_j and W_j = e_j - l_j W_{j-1};
//   3. yhat_j = W_j + zin Hg_j for the next step, and Z += zin.
// The part zin G of every increment is added to v as G_j Z once per
// kFluxEvery32r steps, where the right-hand side is recomputed in flux form
// from v.  Six FP32 operations per row and step: the method's forward and
// backward substitution (an FMA, a multiply and an FMA), two carry
// corrections and the accumulation of v.  The factors l, P, dinv, u, Hg live
// in registers; G and the face weights, used only in the flux steps, in
// shared memory.
//
// Rows are padded to 32 R >= nx + 1 with l = u = dinv = 0, so P = G = Hg = 0
// there, their increments are exactly 0 and v stays 0: the Dirichlet value
// beyond the last row.  Table row nx holds the weight of the right boundary
// face.
#include "common.cuh"

namespace klecgc {

constexpr int kFluxEvery32r = 32;

// Per-sample table: seven FP32 planes of [R][32] (row i = g R + j at index
// j 32 + g): l, P, dinv, u, Hg, wd (the face left of row i), G, then the
// lane totals F_{R-1} ([32]).  F, G, P and Hg are formed in FP64 from the
// FP32-rounded l, dinv and u that the sweeps use, then rounded.
constexpr int kPlanes32r = 7;

__global__ void k_fine_table32r(const FineCoef64* __restrict__ fc, int64_t S, int nx, int R,
                                float* __restrict__ tab) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * 32) return;
    const int64_t s = t >> 5;
    const int g = (int)(t & 31);
    const FineCoef64* c = fc + s * (nx + 1);
    const int64_t plane = (int64_t)R * 32;
    float* T = tab + s * (kPlanes32r * plane + 32);
    double Fd[64], Gd[64];
    double F = 1.0;
    for (int j = 0; j < R; ++j) {
        const int i = g * R + j;
        const float l = i < nx ? (float)c[i].l : 0.f;
        const float dinv = i < nx ? (float)c[i].dinv : 0.f;
        const float u = i + 1 < nx ? (float)(-c[i + 1].wd * c[i].dinv) : 0.f;
        const float wd = i <= nx ? (float)c[i].wd : 0.f;
        F *= -(double)l;
        Fd[j] = F;
        const int64_t o = (int64_t)j * 32 + g;
        T[0 * plane + o] = l;
        T[2 * plane + o] = dinv;
        T[3 * plane + o] = u;
        T[5 * plane + o] = wd;
    }
    T[kPlanes32r * plane + g] = (float)F;
    double G = 1.0, P = 0.0;
    for (int j = R - 1; j >= 0; --j) {
        const int64_t o = (int64_t)j * 32 + g;
        const double u = (double)T[3 * plane + o];
        P = (double)T[2 * plane + o] * Fd[j] - u * P;
        G *= -u;
        Gd[j] = G;
        T[1 * plane + o] = (float)P;
        T[6 * plane + o] = (float)G;
    }
    double H = 0.0;
    for (int j = 0; j < R; ++j) {
        const int64_t o = (int64_t)j * 32 + g;
        H = Gd[j] - (double)T[0 * plane + o] * H;
        T[4 * plane + o] = (float)H;
    }
}

// The flux-form right-hand side of every row of the lane from v (the values
// after this step's update; vl / vr are the neighbours' boundary values, so
// the two rows next to a lane boundary see the same flux through it),
// followed by the local forward sweep into w.
template <int R, bool REACT>
__device__ __forceinline__ void flux_sweep32r(const float (&v)[R], float (&w)[R],
                                              const float (&fl)[R], const float* WD,
                                              int lane, float vl, float vr, float wd_right,
                                              float src, float dt_react) {
    // an opaque offset, so that the compiler re-reads the weights in every
    // flux step instead of holding R of them in registers
    int o0 = lane;
    asm volatile("" : "+r"(o0));
    float fprev = __fmul_rn(WD[o0], __fsub_rn(v[0], vl));
    float y = 0.f;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const float wr = j + 1 < R ? WD[(j + 1) * 32 + o0] : wd_right;
        const float vn = j + 1 < R ? v[j + 1] : vr;
        const float f = __fmul_rn(wr, __fsub_rn(vn, v[j]));
        float rhs = __fsub_rn(f, fprev);
        if (REACT) rhs = __fadd_rn(rhs, __fsub_rn(src, __fmul_rn(dt_react, v[j])));
        y = fmaf(-fl[j], y, rhs);
        w[j] = y;
        fprev = f;
    }
}

// LT intervals per warp in turn (a compile-time count: with LT = 1 the
// interval loop disappears, and with it the registers that the loop keeps
// alive, which at R = 32 is the difference between no spills and some).
// The carry scans are interleaved with the sweeps in program order (a warp
// issues in order): one scan level every SP rows, so that a shuffle's
// latency is covered by independent sweep work.
template <int R, int LT, bool REACT>
__global__ void __launch_bounds__(128) k_fine32r(
    int64_t S, int N, int nx, int J, int cps, float dt_react, float dt_f, int in_mode,
    const double* __restrict__ U64, const float2* __restrict__ Udf, const double* __restrict__ u0,
    const float* __restrict__ c32, const float* __restrict__ tab, float* __restrict__ fout,
    const int* __restrict__ active) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int64_t plane = (int64_t)R * 32;
    constexpr int SP = R >= 12 ? R / 6 : 1;                  // rows per scan level
    constexpr int KIN = R / SP < 5 ? R / SP : 5;             // levels inside the sweep
    // wd and G (read only in the flux steps) staged in shared memory, so
    // that a flux step does not wait for L2
    __shared__ float sWD[R * 32], sG[R * 32];
    const int64_t s = blockIdx.x / cps;
    const int part = (int)(blockIdx.x - s * cps);
    if (!active[s]) return;
    const int nw = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_first = part * nw + warp, n_stride = cps * nw;
    const float* T = tab + s * (kPlanes32r * plane + 32);
    // the register factors first, so that their loads overlap the staging
    float fl[R], fP[R], fd[R], fu[R], fH[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int o = j * 32 + lane;
        fl[j] = __ldg(T + 0 * plane + o);
        fP[j] = __ldg(T + 1 * plane + o);
        fd[j] = __ldg(T + 2 * plane + o);
        fu[j] = __ldg(T + 3 * plane + o);
        fH[j] = __ldg(T + 4 * plane + o);
    }
    for (int e = threadIdx.x; e < R * 32; e += blockDim.x) {
        sWD[e] = __ldg(T + 5 * plane + e);
        sG[e] = __ldg(T + 6 * plane + e);
    }
    __syncthreads();
    if (n_first >= N) return;

    const float wd_right = lane < 31 ? sWD[lane + 1] : 0.f;   // face right of the last row

    // scan multipliers (data independent): products of the lane totals
    float cf[5], cb[5];
    {
        float af = __ldg(T + kPlanes32r * plane + lane), ab = sG[lane];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int d = 1 << k;
            const float pf = __shfl_up_sync(FULL, af, d);
            const float pb = __shfl_down_sync(FULL, ab, d);
            cf[k] = lane >= d ? af : 0.f;
            cb[k] = lane + d <= 31 ? ab : 0.f;
            if (lane >= d) af *= pf;
            if (lane + d <= 31) ab *= pb;
        }
    }
    const int flux_every = in_mode == 0 ? 1 : kFluxEvery32r;
    const float src = in_mode == 0 ? dt_f : 0.f;
    const int64_t sbase = s * (int64_t)nx * N;

#pragma unroll 1
    for (int it = 0; it < LT; ++it) {
        const int n = n_first + it * n_stride;
        if (n >= N) return;
        float v[R], w[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int i = lane * R + j;
            float x0 = 0.f;
            if (i < nx) {
                const int64_t o = sbase + (int64_t)i * N + n - 1;
                if (in_mode == 1)
                    x0 = n > 0 ? c32[o] : 0.f;
                else if (n == 0)
                    x0 = (float)u0[i];
                else
                    x0 = Udf ? Udf[o].x : (float)U64[o];
            }
            v[j] = x0;
        }
        {
            float vl = __shfl_up_sync(FULL, v[R - 1], 1);
            float vr = __shfl_down_sync(FULL, v[0], 1);
            if (lane == 0) vl = 0.f;
            if (lane == 31) vr = 0.f;
            flux_sweep32r<R, REACT>(v, w, fl, sWD, lane, vl, vr, wd_right, src, dt_react);
        }
        float Z = 0.f;   // sum of zin since v last took its G part
        for (int step = 0; step < J; ++step) {
            // 1. forward carry scan (lane totals of yhat) within the local
            //    backward sweep X = xhat(yhat)
            float b = w[R - 1];
            float t = __shfl_up_sync(FULL, b, 1);
            float X = 0.f;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int j = R - 1 - q;
                X = fmaf(-fu[j], X, __fmul_rn(fd[j], w[j]));
                w[j] = X;
                if (q % SP == SP - 1 && q / SP < 5) {
                    const int k = q / SP;
                    b = fmaf(cf[k], t, b);
                    t = __shfl_up_sync(FULL, b, k < 4 ? 2 << k : 1);
                }
            }
#pragma unroll
            for (int k = KIN; k < 5; ++k) {
                b = fmaf(cf[k], t, b);
                t = __shfl_up_sync(FULL, b, k < 4 ? 2 << k : 1);
            }
            const float yin = lane ? t : 0.f;
            // 2. backward carry scan (x at each lane's first row) within
            //    e = X + yin P, v += e, W = fwd(e)
            float z = fmaf(yin, fP[0], w[0]);
            t = __shfl_down_sync(FULL, z, 1);
            float W = 0.f;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const float e = fmaf(yin, fP[j], w[j]);
                v[j] += e;
                W = fmaf(-fl[j], W, e);
                w[j] = W;
                if (j % SP == SP - 1 && j / SP < 5) {
                    const int k = j / SP;
                    z = fmaf(cb[k], t, z);
                    t = __shfl_down_sync(FULL, z, k < 4 ? 2 << k : 1);
                }
            }
#pragma unroll
            for (int k = KIN; k < 5; ++k) {
                z = fmaf(cb[k], t, z);
                t = __shfl_down_sync(FULL, z, k < 4 ? 2 << k : 1);
            }
            const float zin = lane < 31 ? t : 0.f;
            Z += zin;
            // 3. the next step's yhat, or (flux steps) v's G part and the
            //    flux-form right-hand side
            const bool more = step + 1 < J;
            if (more && (step + 1) % flux_every != 0) {
#pragma unroll
                for (int j = 0; j < R; ++j) w[j] = fmaf(zin, fH[j], w[j]);
            } else {
                int o0 = lane;
                asm volatile("" : "+r"(o0));   // re-read G in every flux step
#pragma unroll
                for (int j = 0; j < R; ++j) v[j] = fmaf(sG[j * 32 + o0], Z, v[j]);
                Z = 0.f;
                if (more) {
                    float vl = __shfl_up_sync(FULL, v[R - 1], 1);
                    float vr = __shfl_down_sync(FULL, v[0], 1);
                    if (lane == 0) vl = 0.f;
                    if (lane == 31) vr = 0.f;
                    flux_sweep32r<R, REACT>(v, w, fl, sWD, lane, vl, vr, wd_right, src, dt_react);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int i = lane * R + j;
            if (i < nx) fout[sbase + (int64_t)i * N + n] = v[j];
        }
    }
}

size_t fine_table32r_bytes(int64_t S, int R) {
    return (size_t)S * (kPlanes32r * (size_t)R * 32 + 32) * sizeof(float);
}

void launch_fine_table32r(const FineCoef64* fc, int64_t S, int nx, int R, float* table,
                          cudaStream_t st) {
    if (S == 0) return;
    k_fine_table32r<<<(unsigned)((S * 32 + 127) / 128), 128, 0, st>>>(fc, S, nx, R, table);
}

bool fine32r_supported(int R, int L) {
    return (R == 2 || R == 4 || R == 8 || R == 16 || R == 32) && (L == 1 || L == 4);
}

template <int R, int LT>
static void launch_fine32r_r(int64_t S, int N, int nx, int J, double dt, double react,
                             double forcing, int in_mode, const double* U64, const float2* Udf,
                             const double* u0, const float* c32, const float* table, float* fout,
                             const int* active, cudaStream_t st) {
    constexpr int warps = 4;
    const int cps = (N + warps * LT - 1) / (warps * LT);
    const bool react_terms = react != 0.0 || (forcing != 0.0 && in_mode == 0);
    if (react_terms)
        k_fine32r<R, LT, true><<<(unsigned)(S * cps), warps * 32, 0, st>>>(
            S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0,
            c32, table, fout, active);
    else
        k_fine32r<R, LT, false><<<(unsigned)(S * cps), warps * 32, 0, st>>>(
            S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0,
            c32, table, fout, active);
}

void launch_fine32r(int R, int L, int64_t S, int N, int nx, int J, double dt, double react,
                    double forcing, int in_mode, const double* U64, const float2* Udf,
                    const double* u0, const float* c32, const float* table, float* fout,
                    const int* active, cudaStream_t st) {
    if (S == 0 || !fine32r_supported(R, L)) return;
    switch (R * 10 + L) {
#define KLECGC_F32R(RR, LL)                                                                    \
    case RR * 10 + LL:                                                                         \
        launch_fine32r_r<RR, LL>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32,  \
                                 table, fout, active, st);                                     \
        break;
        KLECGC_F32R(2, 1)
        KLECGC_F32R(4, 1)
        KLECGC_F32R(8, 1)
        KLECGC_F32R(16, 1)
        KLECGC_F32R(32, 1)
        KLECGC_F32R(2, 4)
        KLECGC_F32R(4, 4)
        KLECGC_F32R(8, 4)
        KLECGC_F32R(16, 4)
        KLECGC_F32R(32, 4)
#undef KLECGC_F32R
        default: break;
    }
}

}  // namespace klecgc
