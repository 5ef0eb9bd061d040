// FP32 fine propagator with the LU factors in registers (mixed modes).
//
// The same computation as k_fine32 (J backward-Euler steps of
// M = I + dt(A + cI) per interval, increment form with the flux-form
// right-hand side every kFluxEvery32w steps, two intervals per lane group),
// laid out so that every factor a lane uses lives in its registers for all J
// steps: W warps (32 W lanes) share one pair of intervals, lane g of the
// group owns rows [g R, g R + R) with R <= 16, and holds l, F, dinv, u, G of
// those rows (5 R floats) beside the two intervals' state (4 R floats).
// Where k_fine32 reads the factors from shared memory in every step (20 bytes
// per row and step, which bounded it by shared-memory bandwidth), this kernel
// reads them once.
//
// Per step and interval, as in k_fine32: the local forward sweep of each lane
// from a zero carry, a 5-level shuffle scan of the carries within the warp,
// the forward correction, the diagonal and the local backward sweep, the
// backward scan, and the update v += delta.  Between warps the carries are
// resolved through shared memory: each warp publishes the value its scan
// gives for its last (forward) or first (backward) row with a zero carry into
// the warp, and every warp combines the published values of the warps before
// (after) it with the warp-total multipliers, which are data independent:
//   forward:  c_in(w) = y_out(w-1),  y_out(w) = b_31(w) + TA(w) c_in(w)
//   backward: e_in(w) = z_out(w+1),  z_out(w) = z_0(w) + TB(w) e_in(w)
// so a lane's carry is its in-warp carry plus (product of the multipliers
// between it and the warp boundary) times the warp's carry.  Two barriers per
// step; the values next to a warp boundary that the flux form needs travel
// with the backward carries.
#include "common.cuh"

namespace klecgc {

constexpr int kFluxEvery32w = 16;

// Per-sample table of six FP32 arrays of [R][32 W] (row i = g R + j of lane g
// at index j 32W + g): l (forward multiplier), F = prod_{k<=j} (-l_k) and
// G = prod_{k>=j} (-u_k) within the lane (products of the FP32-rounded
// multipliers, so that they match the sweeps), dinv, u = M_{i,i+1} dinv_i,
// wd = dt a_{i-1/2} / h^2 (the face left of row i; row nx holds the right
// boundary face).  Built from the FP64 factors of k_fine_factors; rows
// i >= nx are padding: l = u = dinv = 0, so they stay zero.
__global__ void k_fine_table32w(const FineCoef64* __restrict__ fc, int64_t S, int nx, int R,
                                int W, float* __restrict__ tab) {
    const int LT = 32 * W;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * LT) return;
    const int64_t s = t / LT;
    const int g = (int)(t - s * LT);
    const FineCoef64* c = fc + s * (nx + 1);
    const int64_t plane = (int64_t)R * LT;
    float* T = tab + s * 6 * plane;
    double F = 1.0;
    for (int j = 0; j < R; ++j) {
        const int i = g * R + j;
        const float l = i < nx ? (float)c[i].l : 0.f;
        const float dinv = i < nx ? (float)c[i].dinv : 0.f;
        const float u = i + 1 < nx ? (float)(-c[i + 1].wd * c[i].dinv) : 0.f;
        const float wd = i <= nx ? (float)c[i].wd : 0.f;
        F *= -(double)l;
        const int64_t o = (int64_t)j * LT + g;
        T[0 * plane + o] = l;
        T[1 * plane + o] = (float)F;
        T[2 * plane + o] = dinv;
        T[3 * plane + o] = u;
        T[5 * plane + o] = wd;
    }
    double G = 1.0;
    for (int j = R - 1; j >= 0; --j) {
        const int64_t o = (int64_t)j * LT + g;
        G *= -(double)T[3 * plane + o];
        T[4 * plane + o] = (float)G;
    }
}

template <int W, int R, bool REACT>
__global__ void __launch_bounds__(32 * W) k_fine32w(
    int64_t S, int N, int nx, int J, int cps, float dt_react, float dt_f, int in_mode,
    const double* __restrict__ U64, const float2* __restrict__ Udf, const double* __restrict__ u0,
    const float* __restrict__ c32, const float* __restrict__ tab, float* __restrict__ fout,
    const int* __restrict__ active) {
    static_assert(R >= 2, "a row next to each lane boundary on both sides");
    constexpr int LT = 32 * W;
    constexpr int64_t plane = (int64_t)R * LT;
    constexpr unsigned FULL = 0xffffffffu;
    // cross-warp carries, double-buffered by step parity: [parity][warp][q]
    __shared__ float sFw[2][W][2], sBw[2][W][2];
    // flux steps: (v + xhat) of each warp's last row, v of its first row
    __shared__ float sVL[W][2], sV0[W][2];
    __shared__ float sTA[W], sTB[W];
    const int64_t s = blockIdx.x / cps;
    const int part = blockIdx.x - (int)(s * cps);
    if (!active[s]) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp * 32 + lane;
    const int n0 = part * 2;
    const float* T = tab + s * 6 * plane;

    float fl[R], fF[R], fd[R], fu[R], fG[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int64_t o = (int64_t)j * LT + g;
        fl[j] = T[0 * plane + o];
        fF[j] = T[1 * plane + o];
        fd[j] = T[2 * plane + o];
        fu[j] = T[3 * plane + o];
        fG[j] = T[4 * plane + o];
    }
    const float* WD = T + 5 * plane;
    const float gprev = g > 0 ? T[4 * plane + (int64_t)(R - 1) * LT + g - 1] : 0.f;  // G_{R-1} of lane g-1
    const float wd_right = g + 1 < LT ? WD[g + 1] : 0.f;                          // face right of the last row

    // scan multipliers within the warp (data independent)
    float cf[5], cb[5];
    float af = fF[R - 1], ab = fG[0];
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
    // af = product of the lane totals of lanes <= lane, ab = of lanes >= lane
    float pa_ex = __shfl_up_sync(FULL, af, 1);     // lanes < lane (the warp carry's multiplier)
    float pb_ex = __shfl_down_sync(FULL, ab, 1);   // lanes > lane
    if (lane == 0) pa_ex = 1.f;
    if (lane == 31) pb_ex = 1.f;
    if (W > 1) {
        if (lane == 31) sTA[warp] = af;
        if (lane == 0) sTB[warp] = ab;
    }

    const int flux_every = in_mode == 0 ? 1 : kFluxEvery32w;
    const float src = in_mode == 0 ? dt_f : 0.f;

    float v[2][R], w[2][R];
    const int64_t sbase = s * (int64_t)nx * N;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int n = n0 + q;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int i = g * R + j;
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
    // neighbour values of the start state across warp boundaries
    if (W > 1) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (lane == 31) sVL[warp][q] = v[q][R - 1];
            if (lane == 0) sV0[warp][q] = v[q][0];
        }
    }
    __syncthreads();
    // step-0 right-hand side (flux form) and local forward sweep
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float vl = __shfl_up_sync(FULL, v[q][R - 1], 1);
        float vr = __shfl_down_sync(FULL, v[q][0], 1);
        if (lane == 0) vl = warp > 0 ? sVL[warp - 1][q] : 0.f;
        if (lane == 31) vr = warp + 1 < W ? sV0[warp + 1][q] : 0.f;
        float fprev = WD[g] * (v[q][0] - vl);
        float yprev = 0.f;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const float wr = (j + 1 < R) ? WD[(int64_t)(j + 1) * LT + g] : wd_right;
            const float vn = (j + 1 < R) ? v[q][j + 1] : vr;
            const float f = wr * (vn - v[q][j]);
            float rhs = f - fprev;
            if (REACT) rhs += src - dt_react * v[q][j];
            yprev = fmaf(-fl[j], yprev, rhs);
            w[q][j] = yprev;
            fprev = f;
        }
    }

    for (int step = 0; step < J; ++step) {
        const int par = step & 1;
        // forward carries: in-warp scan, then the warps before this one
        float yin[2], bl[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float b = w[q][R - 1];
#pragma unroll
            for (int k = 0; k < 5; ++k) b = fmaf(cf[k], __shfl_up_sync(FULL, b, 1 << k), b);
            const float t = __shfl_up_sync(FULL, b, 1);
            yin[q] = lane ? t : 0.f;
            bl[q] = b;
        }
        if (W > 1) {
            if (lane == 31) {
                sFw[par][warp][0] = bl[0];
                sFw[par][warp][1] = bl[1];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float c = 0.f;
#pragma unroll
                for (int u = 0; u < W; ++u)
                    if (u < warp) c = fmaf(sTA[u], c, sFw[par][u][q]);
                yin[q] = fmaf(pa_ex, c, yin[q]);
            }
        }
        // descending: forward correction, diagonal, local backward sweep
        float xn[2] = {0.f, 0.f};
#pragma unroll
        for (int j = R - 1; j >= 0; --j) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float y = fmaf(fF[j], yin[q], w[q][j]);
                const float xh = fmaf(-fu[j], xn[q], y * fd[j]);
                w[q][j] = xh;
                xn[q] = xh;
            }
        }
        const bool more = step + 1 < J;
        const bool flux = !more || (step + 1) % flux_every == 0;
        // backward carries: z = true x at this lane's first row, zin = the
        // next lane's
        float z[2], zin[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float b = w[q][0];
#pragma unroll
            for (int k = 0; k < 5; ++k) b = fmaf(cb[k], __shfl_down_sync(FULL, b, 1 << k), b);
            z[q] = b;
            const float t = __shfl_down_sync(FULL, b, 1);
            zin[q] = lane < 31 ? t : 0.f;
        }
        if (W > 1) {
            if (lane == 0) {
                sBw[par][warp][0] = z[0];
                sBw[par][warp][1] = z[1];
            }
            if (flux) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (lane == 31) sVL[warp][q] = v[q][R - 1] + w[q][R - 1];
                    if (lane == 0) sV0[warp][q] = v[q][0];
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float e = 0.f;
#pragma unroll
                for (int u = W - 1; u >= 0; --u)
                    if (u > warp) e = fmaf(sTB[u], e, sBw[par][u][q]);
                z[q] = fmaf(ab, e, z[q]);
                zin[q] = fmaf(pb_ex, e, zin[q]);
            }
        }
        if (flux) {
            // v += delta, then the next right-hand side in flux form from v
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                // neighbour values after this step's update, for the next rhs;
                // the rows next to a boundary are updated below by exactly
                // the formulas used here, so both sides of a face see the
                // same values and the flux form stays conservative
                float pl = __shfl_up_sync(FULL, v[q][R - 1] + w[q][R - 1], 1);
                float pr = __shfl_down_sync(FULL, v[q][0], 1);
                if (lane == 0) pl = warp > 0 ? sVL[warp - 1][q] : 0.f;
                if (lane == 31) pr = warp + 1 < W ? sV0[warp + 1][q] : 0.f;
                const float vl = g > 0 ? fmaf(gprev, z[q], pl) : 0.f;
                const float vr = g + 1 < LT ? pr + zin[q] : 0.f;
                float fprev = 0.f, yprev = 0.f, lprev = 0.f;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (j == 0)
                        v[q][0] = v[q][0] + z[q];
                    else if (j == R - 1)
                        v[q][R - 1] = fmaf(fG[R - 1], zin[q], v[q][R - 1] + w[q][R - 1]);
                    else
                        v[q][j] += fmaf(fG[j], zin[q], w[q][j]);
                    if (more) {
                        const float f = WD[(int64_t)j * LT + g] * (v[q][j] - (j ? v[q][j - 1] : vl));
                        if (j) {
                            float rhs = f - fprev;
                            if (REACT) rhs += src - dt_react * v[q][j - 1];
                            yprev = fmaf(-lprev, yprev, rhs);
                            w[q][j - 1] = yprev;
                        }
                        fprev = f;
                        lprev = fl[j];
                    }
                }
                if (more) {
                    const float f = wd_right * (vr - v[q][R - 1]);
                    float rhs = f - fprev;
                    if (REACT) rhs += src - dt_react * v[q][R - 1];
                    w[q][R - 1] = fmaf(-lprev, yprev, rhs);
                }
            }
        } else {
            // delta_j = xhat_j + G_j zin, v += delta, and the next step's
            // local forward sweep on the right-hand side delta
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float yprev = 0.f;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    const float d = fmaf(fG[j], zin[q], w[q][j]);
                    v[q][j] += d;
                    yprev = fmaf(-fl[j], yprev, d);
                    w[q][j] = yprev;
                }
            }
        }
    }

    // epilogue: F (in_mode 0) or F0(c) (in_mode 1) for this lane's rows, FP32
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = g * R + j;
        if (i >= nx) break;
        float* o = fout + sbase + (int64_t)i * N + n0;
        if (n0 + 1 < N)
            *reinterpret_cast<float2*>(o) = make_float2(v[0][j], v[1][j]);
        else if (n0 < N)
            o[0] = v[0][j];
    }
}

}  // namespace klecgc

namespace klecgc {

// Launch shape: W warps per pair of intervals, R rows per lane, 32 W R >= nx + 1
// (the padding row carries the right boundary face).  Rule: one warp while
// 16 rows per lane suffice, otherwise 16 rows per lane on 2 or 4 warps.
Fine32wShape fine32w_shape(int nx) {
    const int need = nx + 1;
    for (int R : {2, 4, 8, 16})
        if (32 * R >= need) return {1, R};
    for (int W : {2, 4})
        if (32 * W * 16 >= need) return {W, 16};
    return {0, 0};
}

bool fine32w_supported(Fine32wShape sh) {
    switch (sh.W * 100 + sh.R) {
        case 102: case 104: case 108: case 116: case 208: case 216: case 408: case 416:
            return true;
        default:
            return false;
    }
}

size_t fine_table32w_bytes(int64_t S, Fine32wShape sh) {
    return (size_t)S * 6 * (size_t)sh.R * 32 * sh.W * sizeof(float);
}

void launch_fine_table32w(const FineCoef64* fc, int64_t S, int nx, Fine32wShape sh, float* table,
                          cudaStream_t st) {
    const int64_t n = S * 32 * sh.W;
    if (n == 0) return;
    k_fine_table32w<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(fc, S, nx, sh.R, sh.W, table);
}

template <int W, int R>
static void launch_w(int64_t S, int N, int nx, int J, double dt, double react, double forcing,
                     int in_mode, const double* U64, const float2* Udf, const double* u0,
                     const float* c32, const float* table, float* fout, const int* active,
                     cudaStream_t st) {
    const int cps = (N + 1) / 2;
    const bool react_terms = react != 0.0 || (forcing != 0.0 && in_mode == 0);
    if (react_terms)
        k_fine32w<W, R, true><<<(unsigned)(S * cps), 32 * W, 0, st>>>(
            S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0,
            c32, table, fout, active);
    else
        k_fine32w<W, R, false><<<(unsigned)(S * cps), 32 * W, 0, st>>>(
            S, N, nx, J, cps, (float)(dt * react), (float)(dt * forcing), in_mode, U64, Udf, u0,
            c32, table, fout, active);
}

void launch_fine32w(Fine32wShape sh, int64_t S, int N, int nx, int J, double dt, double react,
                    double forcing, int in_mode, const double* U64, const float2* Udf,
                    const double* u0, const float* c32, const float* table, float* fout,
                    const int* active, cudaStream_t st) {
    if (S == 0) return;
    switch (sh.W * 100 + sh.R) {
#define KLECGC_F32W(WW, RR)                                                                   \
    case WW * 100 + RR:                                                                       \
        launch_w<WW, RR>(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table,  \
                         fout, active, st);                                                    \
        break;
        KLECGC_F32W(1, 2)
        KLECGC_F32W(1, 4)
        KLECGC_F32W(1, 8)
        KLECGC_F32W(1, 16)
        KLECGC_F32W(2, 8)
        KLECGC_F32W(2, 16)
        KLECGC_F32W(4, 8)
        KLECGC_F32W(4, 16)
#undef KLECGC_F32W
        default: break;
    }
}

}  // namespace klecgc

namespace klecgc {

// Every supported shape that covers nx + 1 rows without a wasted doubling
// (32 W R >= nx + 1 > 16 W R): the candidates the autotuner times.
std::vector<Fine32wShape> fine32w_candidates(int nx) {
    std::vector<Fine32wShape> out;
    for (Fine32wShape sh : {Fine32wShape{1, 2}, Fine32wShape{1, 4}, Fine32wShape{1, 8},
                            Fine32wShape{1, 16}, Fine32wShape{2, 8}, Fine32wShape{2, 16},
                            Fine32wShape{4, 8}, Fine32wShape{4, 16}}) {
        const int rows = 32 * sh.W * sh.R;
        if (rows >= nx + 1 && (sh.R == 2 || rows / 2 < nx + 1)) out.push_back(sh);
    }
    return out;
}

}  // namespace klecgc

namespace klecgc {

void launch_fine_any(Fine32wShape sh, int64_t S, int N, int nx, int J, double dt, double react,
                     double forcing, int in_mode, const double* U64, const float2* Udf,
                     const double* u0, const float* c32, const float* table, float* fout,
                     const int* active, cudaStream_t st) {
    if (sh.P)
        launch_fine32p(sh.R, S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table,
                       fout, active, st);
    else if (sh.L)
        launch_fine32r(sh.R, sh.L, S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32,
                       table, fout, active, st);
    else if (sh.W == 0)
        launch_fine32(S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table, fout,
                      active, st);
    else
        launch_fine32w(sh, S, N, nx, J, dt, react, forcing, in_mode, U64, Udf, u0, c32, table,
                       fout, active, st);
}

}  // namespace klecgc
