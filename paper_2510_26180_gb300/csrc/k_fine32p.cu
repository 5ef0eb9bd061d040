// FP32 fine propagator, one interval per warp, factors in registers, each
// lane's R rows split into two halves whose sweeps advance together in packed
// FP32x2 arithmetic (mixed modes).
//
// The computation is the one of k_fine32r (J backward-Euler steps of
// M = I + dt(A + cI) per interval in increment form, the right-hand side in
// flux form from v every kFluxEvery32p steps and in every step on start
// values, the partitioned LU solve regrouped as x = X + yin P + zin G with
// the next forward sweep fwd(X + yin P) + zin Hg), with one change of
// partition: lane g owns rows [g R, g R + R) as two halves of H = R / 2 rows,
// A = [g R, g R + H) and B = [g R + H, g R + R), and every per-row quantity
// of the lane is a pair (row g R + j of A, row g R + H + j of B).  The local
// sweeps of A and B are independent, so one FFMA2 advances both: a step's
// backward sweep, correction, accumulation and forward sweep take H packed
// instructions each instead of R scalar ones, and the sweeps' dependent
// chains are half as long.
//
// The warp scans see one affine map per lane.  Forward: with yhat the local
// sweeps (zero carry into each half) and F_A, F_B the half products of -l,
//   y_B,end = yhat_B,end + F_B (yhat_A,end + F_A yin_A) = b + (F_A F_B) yin_A,
// so the scan runs on b with the lane multiplier F_A F_B, and after it
// yin_B = yhat_A,end + F_A yin_A.  Backward: with z_A, z_B the first-row
// values X_0 + yin P_0 of each half and G_A, G_B the half products of -u,
//   x_A,first = z_A + G_A (z_B + G_B zin_B) = z + (G_A G_B) zin_B,
// and after the scan zin_A = z_B + G_B zin_B.
//
// Rows are padded to 32 R >= nx + 1 with l = u = dinv = 0, as in k_fine32r.
#include "common.cuh"

namespace klecgc {

constexpr int kFluxEvery32p = 32;

// Per-sample table: seven planes of [H][32] float2 (pair j of lane g at
// index j 32 + g; .x half A, .y half B): -l, P, dinv, -u, Hg, wd (the face
// left of the row), G; then [32] float2 of the half products F_A, F_B.  F, G,
// P and Hg are formed per half in FP64 from the FP32-rounded l, dinv and u
// that the sweeps use, then rounded.  l and u are stored negated, so that the
// packed sweeps need no negation.
constexpr int kPlanes32p = 7;

size_t fine_table32p_bytes(int64_t S, int R) {
    return (size_t)S * (kPlanes32p * (size_t)(R / 2) * 32 + 32) * sizeof(float2);
}

bool fine32p_supported(int R) { return R == 4 || R == 8 || R == 16 || R == 32; }

// One thread per half (two per lane).
__global__ void k_fine_table32p(const FineCoef64* __restrict__ fc, int64_t S, int nx, int R,
                                float2* __restrict__ tab) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * 64) return;
    const int64_t s = t >> 6;
    const int g = (int)(t & 63) >> 1, half = (int)(t & 1);
    const int H = R / 2;
    const FineCoef64* c = fc + s * (nx + 1);
    const int64_t plane = (int64_t)H * 32;
    float* T = reinterpret_cast<float*>(tab + s * (kPlanes32p * plane + 32));
    auto at = [&](int p, int j) -> float& {
        return T[2 * (p * plane + (int64_t)j * 32 + g) + half];
    };
    double Fd[16], Gd[16];
    float lf[16], uf[16];
    double F = 1.0;
    for (int j = 0; j < H; ++j) {
        const int i = g * R + half * H + j;
        const float l = i < nx ? (float)c[i].l : 0.f;
        const float dinv = i < nx ? (float)c[i].dinv : 0.f;
        const float u = i + 1 < nx ? (float)(-c[i + 1].wd * c[i].dinv) : 0.f;
        lf[j] = l;
        uf[j] = u;
        F *= -(double)l;
        Fd[j] = F;
        at(0, j) = -l;
        at(2, j) = dinv;
        at(3, j) = -u;
        at(5, j) = i <= nx ? (float)c[i].wd : 0.f;
    }
    T[2 * (kPlanes32p * plane + g) + half] = (float)F;
    double G = 1.0, P = 0.0;
    for (int j = H - 1; j >= 0; --j) {
        const double u = (double)uf[j];
        P = (double)at(2, j) * Fd[j] - u * P;
        G *= -u;
        Gd[j] = G;
        at(1, j) = (float)P;
        at(6, j) = (float)G;
    }
    double Hh = 0.0;
    for (int j = 0; j < H; ++j) {
        Hh = Gd[j] - (double)lf[j] * Hh;
        at(4, j) = (float)Hh;
    }
}

// The flux-form right-hand side of the lane's rows from v (vl / vr: the
// neighbouring lanes' boundary values) and the local forward sweep of each
// half into w.  Scalar: it runs once in kFluxEvery32p steps, and FP32x2 has
// no packed subtraction.
template <int H, bool REACT>
__device__ __forceinline__ void flux_sweep32p(const float2 (&v)[H], float2 (&w)[H],
                                              const float2 (&nl)[H], const float2* WD, int lane,
                                              float vl, float vr, float wd_right, float src,
                                              float dt_react) {
    // an opaque offset, so that the weights are re-read in every flux step
    // instead of being held in registers
    int o0 = lane;
    asm volatile("" : "+r"(o0));
    const float2 wd0 = WD[o0];
    float fpa = __fmul_rn(wd0.x, __fsub_rn(v[0].x, vl));
    float fpb = __fmul_rn(wd0.y, __fsub_rn(v[0].y, v[H - 1].x));
    float ya = 0.f, yb = 0.f;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float wra, wrb, vna, vnb;
        if (j + 1 < H) {
            const float2 wr = WD[(j + 1) * 32 + o0];
            wra = wr.x;
            wrb = wr.y;
            vna = v[j + 1].x;
            vnb = v[j + 1].y;
        } else {   // A's last row faces B's first; B's last the next lane
            wra = wd0.y;
            wrb = wd_right;
            vna = v[0].y;
            vnb = vr;
        }
        const float fa = __fmul_rn(wra, __fsub_rn(vna, v[j].x));
        const float fb = __fmul_rn(wrb, __fsub_rn(vnb, v[j].y));
        float ra = __fsub_rn(fa, fpa), rb = __fsub_rn(fb, fpb);
        if (REACT) {
            ra = __fadd_rn(ra, __fsub_rn(src, __fmul_rn(dt_react, v[j].x)));
            rb = __fadd_rn(rb, __fsub_rn(src, __fmul_rn(dt_react, v[j].y)));
        }
        ya = fmaf(nl[j].x, ya, ra);
        yb = fmaf(nl[j].y, yb, rb);
        w[j] = make_float2(ya, yb);
        fpa = fa;
        fpb = fb;
    }
}

// One interval per warp.  The carry scans are interleaved with the sweeps in
// program order, one scan level every SP pairs.
template <int R, bool REACT>
__global__ void __launch_bounds__(128) k_fine32p(
    int64_t S, int N, int nx, int J, int cps, float dt_react, float dt_f, int in_mode,
    const double* __restrict__ U64, const float2* __restrict__ Udf, const double* __restrict__ u0,
    const float* __restrict__ c32, const float2* __restrict__ tab, float* __restrict__ fout,
    const int* __restrict__ active) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int H = R / 2;
    constexpr int64_t plane = (int64_t)H * 32;
    constexpr int SP = H >= 10 ? H / 5 : 1;
    constexpr int KIN = H / SP < 5 ? H / SP : 5;
    // wd and G (read only in the flux steps) staged in shared memory
    __shared__ float2 sWD[H * 32], sG[H * 32];
    const int64_t s = blockIdx.x / cps;
    const int part = (int)(blockIdx.x - s * cps);
    if (!active[s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = part * (blockDim.x >> 5) + warp;
    const float2* T = tab + s * (kPlanes32p * plane + 32);
    float2 nl[H], fP[H], fd[H], nu[H], fH[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const int o = j * 32 + lane;
        nl[j] = __ldg(T + 0 * plane + o);
        fP[j] = __ldg(T + 1 * plane + o);
        fd[j] = __ldg(T + 2 * plane + o);
        nu[j] = __ldg(T + 3 * plane + o);
        fH[j] = __ldg(T + 4 * plane + o);
    }
    for (int e = threadIdx.x; e < H * 32; e += blockDim.x) {
        sWD[e] = __ldg(T + 5 * plane + e);
        sG[e] = __ldg(T + 6 * plane + e);
    }
    __syncthreads();
    if (n >= N) return;

    const float wd_right = lane < 31 ? sWD[lane + 1].x : 0.f;   // face right of the last row
    const float2 Ft = __ldg(T + kPlanes32p * plane + lane);      // F_A, F_B
    const float2 G0 = sG[lane];                                   // G_A, G_B
    // scan multipliers (data independent): products of the lane maps
    float cf[5], cb[5];
    {
        float af = Ft.x * Ft.y, ab = G0.x * G0.y;
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
    const int flux_every = in_mode == 0 ? 1 : kFluxEvery32p;
    const float src = in_mode == 0 ? dt_f : 0.f;
    const int64_t sbase = s * (int64_t)nx * N;

    float2 v[H], w[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float x0[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane * R + h * H + j;
            float x = 0.f;
            if (i < nx) {
                const int64_t o = sbase + (int64_t)i * N + n - 1;
                if (in_mode == 1)
                    x = n > 0 ? c32[o] : 0.f;
                else if (n == 0)
                    x = (float)u0[i];
                else
                    x = Udf ? Udf[o].x : (float)U64[o];
            }
            x0[h] = x;
        }
        v[j] = make_float2(x0[0], x0[1]);
    }
    {
        float vl = __shfl_up_sync(FULL, v[H - 1].y, 1);
        float vr = __shfl_down_sync(FULL, v[0].x, 1);
        if (lane == 0) vl = 0.f;
        if (lane == 31) vr = 0.f;
        flux_sweep32p<H, REACT>(v, w, nl, sWD, lane, vl, vr, wd_right, src, dt_react);
    }
    float2 Z = make_float2(0.f, 0.f);   // sums of zin since v last took its G part
    for (int step = 0; step < J; ++step) {
        // 1. forward carry scan of the lane maps, within the local backward
        //    sweeps X = xhat(yhat) of both halves
        const float ya_end = w[H - 1].x;
        float b = fmaf(Ft.y, ya_end, w[H - 1].y);
        float t = __shfl_up_sync(FULL, b, 1);
        float2 X = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const int j = H - 1 - q;
            X = __ffma2_rn(nu[j], X, __fmul2_rn(fd[j], w[j]));
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
        const float yin_a = lane ? t : 0.f;
        const float2 yin = make_float2(yin_a, fmaf(Ft.x, yin_a, ya_end));
        // 2. backward carry scan of the lane maps, within e = X + yin P,
        //    v += e and W = fwd(e)
        const float zb = fmaf(yin.y, fP[0].y, w[0].y);
        float z = fmaf(G0.x, zb, fmaf(yin.x, fP[0].x, w[0].x));
        t = __shfl_down_sync(FULL, z, 1);
        float2 W = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const float2 e = __ffma2_rn(yin, fP[j], w[j]);
            v[j] = __fadd2_rn(v[j], e);
            W = __ffma2_rn(nl[j], W, e);
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
        const float zin_b = lane < 31 ? t : 0.f;
        const float2 zin = make_float2(fmaf(G0.y, zin_b, zb), zin_b);
        Z = __fadd2_rn(Z, zin);
        // 3. the next step's yhat, or (flux steps) v's G part and the
        //    flux-form right-hand side
        const bool more = step + 1 < J;
        if (more && (step + 1) % flux_every != 0) {
#pragma unroll
            for (int j = 0; j < H; ++j) w[j] = __ffma2_rn(zin, fH[j], w[j]);
        } else {
            int o0 = lane;
            asm volatile("" : "+r"(o0));   // re-read G in every flux step
#pragma unroll
            for (int j = 0; j < H; ++j) v[j] = __ffma2_rn(sG[j * 32 + o0], Z, v[j]);
            Z = make_float2(0.f, 0.f);
            if (more) {
                float vl = __shfl_up_sync(FULL, v[H - 1].y, 1);
                float vr = __shfl_down_sync(FULL, v[0].x, 1);
                if (lane == 0) vl = 0.f;
                if (lane == 31) vr = 0.f;
                flux_sweep32p<H, REACT>(v, w, nl, sWD, lane, vl, vr, wd_right, src, dt_react);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = lane * R + h * H + j;
            if (i < nx) fout[sbase + (int64_t)i * N + n] = h ? v[j].y : v[j].x;
        }
    }
}

void launch_fine_table32p(const FineCoef64* fc, int64_t S, int nx, int R, float* table,
                          cudaStream_t st) {
    if (S == 0 || !fine32p_supported(R)) return;
    k_fine_table32p<<<(unsigned)((S * 64 + 127) / 128), 128, 0, st>>>(
        fc, S, nx, R, reinterpret_cast<float2*>(table));
}

template <int R>
static void launch_fine32p_r(int64_t S, int N, int nx, int J, double dt, double react,
                             double forcing, int in_mode, const double* U64, const float2* Udf,
                             const double* u0, const float* c32, const float* table, float* fout,
                             const int* active, cudaStream_t st) {
    constexpr int warps = 4;
    const int cps = (N + warps - 1) / warps;
    const bool react_terms = react != 0.0 || (forcing != 0.0 && in_mode == 0);
    const float2* tab = reinterpret_cast<const float2*>(table);
    if (react_terms)
        k_fine32p<R, true><<<(unsigned)(S * cps), warps * 32, 0, st>>>(
            S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0,
            c32, tab, fout, active);
    else
        k_fine32p<R, false><<<(unsigned)(S * cps), warps * 32, 0, st>>>(
            S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0,
            c32, tab, fout, active);
}

void launch_fine32p(int R, int64_t S, int N, int nx, int J, double dt, double react,
                    double forcing, int in_mode, const double* U64, const float2* Udf,
                    const double* u0, const float* c32, const float* table, float* fout,
                    const int* active, cudaStream_t st) {
    if (S == 0) return;
    switch (R) {
        case 4: launch_fine32p_r<4>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table, fout, active, st); break;
        case 8: launch_fine32p_r<8>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table, fout, active, st); break;
        case 16: launch_fine32p_r<16>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table, fout, active, st); break;
        case 32: launch_fine32p_r<32>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table, fout, active, st); break;
        default: break;
    }
}

}  // namespace klecgc
