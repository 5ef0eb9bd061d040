// Nonlinear 1D problems and the nonlinear coarse grid correction by
// simplified Newton (Section 3.2, eqs. Newton, Jac, Newton2).  A is the
// flux-form operator with face weights wf_i = a_{i-1/2} / h^2.
//
//   kind 1 (Allen-Cahn-type):  f(u) = -A u - c (u^3 - u) + f0,
//                              grad f(u) = -A - c diag(3 u^2 - 1);
//   kind 2 (Burgers-type):     f(u) = -A u - c conv(u) + f0, the convection
//       (u^2/2)_x in conservative upwind form with the Engquist-Osher flux
//       splitting (Section 5, Burgers equation: upwind convection, central
//       diffusion):  conv(u)_i = (Phi(u_i, u_{i+1}) - Phi(u_{i-1}, u_i)) / h,
//       Phi(l, r) = max(l, 0)^2 / 2 + min(r, 0)^2 / 2, zero boundary values;
//       -grad f(u) = A + (c/h) tridiag(-max(u_{i-1}, 0), |u_i|, min(u_{i+1}, 0)).
//
// Backward Euler (both propagators): one step of size dt solves
//     w - dt f(w) = v   (w + dt A w + dt (nonlinear term) = v + dt f0)
// by Newton's method from w = v: the Jacobian I - dt grad f(w) is tridiagonal
// and factored anew in every Newton iteration (Thomas), stopping when
// max |dw| <= 1e-14 max(1, max |w|) (at most kNewtonMax iterations; a step that
// reaches the cap sets the sample's flag).
//
// CGC: eq. matrix_NT, (C_alpha (x) I) u = dT F(u) + b, F(u)_n = f(U_n - b_n), by
// simplified Newton steps from u_0 = U^k:
//     Jbar u_{l+1} = dT (I (x) K) u_l + dT F(u_l) + b,  K = -gradf_bar,
// gradf_bar = (1/N) sum_n grad f(U_{n,l} - b_n) (eq. Jac), Jbar = C_alpha (x) I +
// dT I (x) K: the linear three steps with shifted factors of K.  Kind 1:
// K = A + diag(e), e_i = c (3 m_i - 1), m_i = mean_n (U_{n,i} - b_{n,i})^2
// (k_nl_prep).  Kind 2: K is a non-symmetric tridiagonal written with face
// couplings (dT-scaled), row i: -lo_i u_{i-1} + (up_i + lo_{i+1}) u_i -
// up_{i+1} u_{i+1}, lo_i = dT (wf_i + (c/h) mean_n max(z_{i-1}, 0)),
// up_i = dT (wf_i - (c/h) mean_n min(z_i, 0)), z = U - b (k_nl_prep_burgers;
// k_cgc_factors_faces factors lambda_k I + dT K from them).
//
// Layout: U, b, rhs [S][nx][N]; columns (s, n) are strided by N (a warp of
// consecutive n coalesces).
#include "common.cuh"

namespace klecgc {

namespace {

constexpr int kNewtonMax = 50;

__device__ __forceinline__ double eo_flux(double l, double r) {
    const double p = fmax(l, 0.0), m = fmin(r, 0.0);
    return 0.5 * (p * p + m * m);
}

// One Newton backward-Euler step on the column w (stride st): v is the start
// value (overwritten by nothing), w the iterate (in/out), cp / dp Thomas
// scratch.  wf: face weights a/h^2 (nx + 1), dt, c (KIND 1: the cubic
// coefficient; KIND 2: c/h), f0.  Returns false if the iteration cap was
// reached; adds the Newton iterations taken to *its.
template <int KIND>
__device__ bool newton_be(int nx, const double* __restrict__ wf, double dt, double c,
                          double f0, const double* v, double* w, double* cp, double* dp,
                          int64_t st, unsigned long long* its) {
    for (int it = 0; it < kNewtonMax; ++it) {
        ++*its;
        // residual R = w - dt f(w) - v and the Thomas forward elimination of
        // (I - dt grad f(w)) d = R, row i: lower d_{i-1} + diag d_i + upper d_{i+1}
        double wl = 0.0, wi = w[0], prevc = 0.0, prevd = 0.0;
        for (int i = 0; i < nx; ++i) {
            const double wr = i + 1 < nx ? w[(int64_t)(i + 1) * st] : 0.0;
            const double fl = dt * wf[i], fr = dt * wf[i + 1];
            const double Aw = fl * (wi - wl) - fr * (wr - wi);          // dt A w
            double R, diag, lower, upper;
            if (KIND == 1) {
                R = wi + Aw + dt * c * (wi * wi * wi - wi) - v[(int64_t)i * st] - dt * f0;
                diag = 1.0 + fl + fr + dt * c * (3.0 * wi * wi - 1.0);
                lower = -fl;
                upper = -fr;
            } else {
                const double dc = dt * c;
                R = wi + Aw + dc * (eo_flux(wi, wr) - eo_flux(wl, wi)) - v[(int64_t)i * st] -
                    dt * f0;
                diag = 1.0 + fl + fr + dc * fabs(wi);
                lower = -fl - dc * fmax(wl, 0.0);
                upper = -fr + dc * fmin(wr, 0.0);
            }
            const double den = diag - lower * prevc;                 // pivot
            const double ci = upper / den;                           // c'_i
            const double di = (R - lower * prevd) / den;
            cp[(int64_t)i * st] = ci;
            dp[(int64_t)i * st] = di;
            prevc = ci;
            prevd = di;
            wl = wi;
            wi = wr;
        }
        // back substitution and update, max |d| and max |w|
        double dnext = 0.0, dmax = 0.0, wmax = 0.0;
        for (int i = nx - 1; i >= 0; --i) {
            const double d = dp[(int64_t)i * st] - cp[(int64_t)i * st] * dnext;
            dnext = d;
            const double wn = w[(int64_t)i * st] - d;
            w[(int64_t)i * st] = wn;
            dmax = fmax(dmax, fabs(d));
            wmax = fmax(wmax, fabs(wn));
        }
        if (dmax <= 1e-14 * fmax(1.0, wmax)) return true;
        if (!(dmax == dmax)) return false;
    }
    return false;
}

}  // namespace

// F (J steps of dt = dT/J from start_n = u0 or U_{n-1}) and, with jump set,
// the jump b_n = F_n - G(prev_n), prev_1 = alpha U_N, prev_n = U_{n-1}, per
// column (s, n); without it bout receives F.  Scratch: v, cp, dp, g [S][nx][N].
template <int KIND>
__global__ void __launch_bounds__(128) k_fine_newton(
    int64_t S, int N, int nx, int J, double dT, double alpha, double c, double f0, int jump,
    const double* __restrict__ U, const double* __restrict__ u0, const double* __restrict__ wf,
    double* __restrict__ bout, double* __restrict__ vs, double* __restrict__ cps,
    double* __restrict__ dps, double* __restrict__ gs, const int* __restrict__ active,
    int* __restrict__ ifail, unsigned long long* __restrict__ itcount) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t s = t / N;
    const int n = (int)(t - s * N);
    if (s >= S || !active[s]) return;
    const int64_t base = s * (int64_t)nx * N + n;
    const double* Us = U + s * (int64_t)nx * N;
    const double* wfs = wf + s * (nx + 1);
    double* w = bout + base;
    double* v = vs + base;
    double* cp = cps + base;
    double* dp = dps + base;
    bool ok = true;
    unsigned long long its = 0;
    for (int i = 0; i < nx; ++i) w[(int64_t)i * N] = n == 0 ? u0[i] : Us[(int64_t)i * N + n - 1];
    const double dt = dT / J;
    for (int j = 0; j < J && ok; ++j) {
        for (int i = 0; i < nx; ++i) v[(int64_t)i * N] = w[(int64_t)i * N];
        ok = newton_be<KIND>(nx, wfs, dt, c, f0, v, w, cp, dp, N, &its);
    }
    if (jump) {
        // G(prev): one step of dT from prev (start v, iterate g); F stays in w
        double* g = gs + base;
        for (int i = 0; i < nx; ++i) {
            const double pv =
                n == 0 ? alpha * Us[(int64_t)i * N + N - 1] : Us[(int64_t)i * N + n - 1];
            v[(int64_t)i * N] = pv;
            g[(int64_t)i * N] = pv;
        }
        if (ok) ok = newton_be<KIND>(nx, wfs, dT, c, f0, v, g, cp, dp, N, &its);
        for (int i = 0; i < nx; ++i) w[(int64_t)i * N] -= g[(int64_t)i * N];
    }
    if (!ok) ifail[s] = 1;
    if (itcount) atomicAdd(itcount, its);
}

// ---- G lanes per column
// The same Newton backward-Euler steps with each column's rows split over G
// lanes (lane g holds rows [g R, g R + R) of w and v in registers).  The
// tridiagonal Newton system (I - dt grad f(w)) d = R of every iteration is
// solved by the Thomas recurrences, each one split at the lane boundaries
// and joined by a scan over the G lanes:
//   pivots      piv_i = diag_i - lower_i upper_{i-1} / piv_{i-1}, a continued
//               fraction: (p_i, q_i) = (diag_i p_{i-1} - lower_i upper_{i-1}
//               q_{i-1}, p_{i-1}), piv = p / q; the lanes' 2 x 2 products are
//               scanned (rescaled by powers of two, which is exact);
//   forward     y_i = R_i - (lower_i / piv_{i-1}) y_{i-1}, affine maps scanned;
//   backward    d_i = (y_i - upper_i d_{i+1}) / piv_i, affine maps scanned from
//               the right.
// One thread per column left the GPU with S N threads in all (8,192 for 256
// samples x 32 intervals, under two warps per SM) and each of them a chain of
// dependent FP64 operations; G lanes per column give G times the threads and
// a chain G times shorter, for about twice the FP64 operations.  A Newton
// iteration ends for the whole column at once (the lanes share max |d| and
// max |w|); columns of one warp that converged earlier keep their w while
// the others iterate.  Rows beyond nx are identity rows (d = 0, w = 0).
namespace {

__device__ __forceinline__ void m2_rescale(double& a, double& b, double& c, double& d) {
    const double mx = fmax(fmax(fabs(a), fabs(b)), fmax(fabs(c), fabs(d)));
    if (mx > 0.0 && (mx > 0x1p+64 || mx < 0x1p-64)) {
        const int e = ilogb(mx);
        a = scalbn(a, -e);
        b = scalbn(b, -e);
        c = scalbn(c, -e);
        d = scalbn(d, -e);
    }
}

// One Newton backward-Euler step of the column held by this lane group:
// w (in/out) the iterate, v the start value.  Returns false where the
// column's Newton iteration reached the cap or produced a non-finite step.
template <int KIND, int G, int R>
__device__ __forceinline__ bool newton_be_g(int nx, int g, const double (&wfv)[R + 1], double dt, double c,
                            double f0, const double (&v)[R], double (&w)[R], unsigned long long* its) {
    constexpr unsigned FULL = 0xffffffffu;
    bool done = false, ok = true;
    for (int it = 0; it < kNewtonMax; ++it) {
        if (__all_sync(FULL, done)) break;
        if (!done) ++*its;
        double Rr[R], lo[R], up[R], ipv[R];
        // residual and Jacobian rows; w beyond the grid is 0
        double wprev = __shfl_up_sync(FULL, w[R - 1], 1, G);
        double wnext = __shfl_down_sync(FULL, w[0], 1, G);
        if (g == 0) wprev = 0.0;
        if (g == G - 1) wnext = 0.0;
        double dg[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int i = g * R + j;
            const double wi = w[j];
            const double wl = j > 0 ? w[j - 1] : wprev;
            const double wr = j + 1 < R ? w[j + 1] : wnext;
            if (i < nx) {
                const double fl = dt * wfv[j], fr = dt * wfv[j + 1];
                const double Aw = fl * (wi - wl) - fr * (wr - wi);
                if (KIND == 1) {
                    Rr[j] = wi + Aw + dt * c * (wi * wi * wi - wi) - v[j] - dt * f0;
                    dg[j] = 1.0 + fl + fr + dt * c * (3.0 * wi * wi - 1.0);
                    lo[j] = -fl;
                    up[j] = -fr;
                } else {
                    const double dc = dt * c;
                    Rr[j] = wi + Aw + dc * (eo_flux(wi, wr) - eo_flux(wl, wi)) - v[j] - dt * f0;
                    dg[j] = 1.0 + fl + fr + dc * fabs(wi);
                    lo[j] = -fl - dc * fmax(wl, 0.0);
                    up[j] = -fr + dc * fmin(wr, 0.0);
                }
            } else {
                Rr[j] = 0.0;
                dg[j] = 1.0;
                lo[j] = 0.0;
                up[j] = 0.0;
            }
        }
        // pivots: the lane's product of the maps M_i = [[dg_i, -lo_i up_{i-1}], [1, 0]]
        double upl = __shfl_up_sync(FULL, up[R - 1], 1, G);   // up of the row before the lane
        if (g == 0) upl = 0.0;
        double t00 = 1.0, t01 = 0.0, t10 = 0.0, t11 = 1.0;
        {
            // R <= 8 factors with entries ~1 + 2 dt a / h^2 stay inside the
            // FP64 range unless dt a / h^2 exceeds ~1e30, so the lane's
            // product is rescaled once, at its end
            double upp = upl;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double cc = -lo[j] * upp;
                const double n00 = dg[j] * t00 + cc * t10, n01 = dg[j] * t01 + cc * t11;
                t10 = t00;
                t11 = t01;
                t00 = n00;
                t01 = n01;
                upp = up[j];
            }
            m2_rescale(t00, t01, t10, t11);
        }
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const double b00 = __shfl_up_sync(FULL, t00, d, G), b01 = __shfl_up_sync(FULL, t01, d, G);
            const double b10 = __shfl_up_sync(FULL, t10, d, G), b11 = __shfl_up_sync(FULL, t11, d, G);
            if (g >= d) {
                const double n00 = t00 * b00 + t01 * b10, n01 = t00 * b01 + t01 * b11;
                const double n10 = t10 * b00 + t11 * b10, n11 = t10 * b01 + t11 * b11;
                t00 = n00;
                t01 = n01;
                t10 = n10;
                t11 = n11;
                m2_rescale(t00, t01, t10, t11);
            }
        }
        const double pp = __shfl_up_sync(FULL, t00, 1, G), qq = __shfl_up_sync(FULL, t10, 1, G);
        // 1 / (pivot of the row before the lane); one division per row below
        double iprev = (g > 0 && pp != 0.0) ? qq / pp : 1.0;
        {
            double upp = upl;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const double m = lo[j] * iprev;   // multiplier of row j (unused at the first row)
                iprev = 1.0 / (dg[j] - m * upp);
                ipv[j] = iprev;
                lo[j] = m;                        // lo now holds the multipliers
                upp = up[j];
            }
        }
        // forward: y_j = R_j - m_j y_{j-1}; the lane as y_out = a y_in + b
        double a = 1.0, b = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            a = -lo[j] * a;
            b = Rr[j] - lo[j] * b;
        }
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const double pa = __shfl_up_sync(FULL, a, d, G), pb = __shfl_up_sync(FULL, b, d, G);
            if (g >= d) {
                b = fma(a, pb, b);
                a *= pa;
            }
        }
        double y = __shfl_up_sync(FULL, b, 1, G);
        if (g == 0) y = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            y = Rr[j] - lo[j] * y;
            Rr[j] = y;                          // Rr now holds y
        }
        // backward: d_j = (y_j - up_j d_{j+1}) / piv_j; the lane as d_first = C d_in + E
        double C = 1.0, E = 0.0;
#pragma unroll
        for (int j = R - 1; j >= 0; --j) {
            const double cj = -up[j] * ipv[j], ej = Rr[j] * ipv[j];
            E = fma(cj, E, ej);
            C = cj * C;
        }
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const double nc = __shfl_down_sync(FULL, C, d, G), ne = __shfl_down_sync(FULL, E, d, G);
            if (g + d < G) {
                E = fma(C, ne, E);
                C *= nc;
            }
        }
        double dn = __shfl_down_sync(FULL, E, 1, G);
        if (g == G - 1) dn = 0.0;
        double dmax = 0.0, wmax = 0.0;
#pragma unroll
        for (int j = R - 1; j >= 0; --j) {
            const double dj = (Rr[j] - up[j] * dn) * ipv[j];
            dn = dj;
            const double wn = done ? w[j] : w[j] - dj;
            if (!done) w[j] = wn;
            dmax = fmax(dmax, fabs(dj));
            wmax = fmax(wmax, fabs(wn));
        }
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            dmax = fmax(dmax, __shfl_xor_sync(FULL, dmax, d, G));
            wmax = fmax(wmax, __shfl_xor_sync(FULL, wmax, d, G));
        }
        if (!done) {
            if (!(dmax == dmax)) {
                ok = false;
                done = true;
            } else if (dmax <= 1e-14 * fmax(1.0, wmax)) {
                done = true;
            }
        }
    }
    return ok && done;
}

// mode 0: F per column (s, n) (and with jump, b = F - G(prev)) as
// k_fine_newton; mode 1: the sequential fine solution per sample s, written
// every J steps (as k_sequential_newton).
template <int KIND, int G, int R>
__global__ void __launch_bounds__(128) k_newton_g(
    int64_t S, int N, int nx, int J, double dT, double alpha, double c, double f0, int jump,
    int mode, const double* __restrict__ U, const double* __restrict__ u0,
    const double* __restrict__ wf, double* __restrict__ out, const int* __restrict__ active,
    int* __restrict__ ifail, unsigned long long* __restrict__ itcount) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t col = t / G;
    const int g = (int)(t - col * G);
    const int64_t ncol = mode == 0 ? S * N : S;
    // whole warps stay for the shuffles; a group past the end works on
    // a copy of the last column and writes nothing
    const bool real = col < ncol;
    const int64_t cc = real ? col : ncol - 1;
    const int64_t s = mode == 0 ? cc / N : cc;
    const int n = mode == 0 ? (int)(cc - s * N) : 0;
    const bool act = active == nullptr || active[s];
    if (!__any_sync(0xffffffffu, real && act)) return;   // the whole warp is idle
    double wfv[R + 1];
#pragma unroll
    for (int j = 0; j <= R; ++j) {
        const int i = g * R + j;
        wfv[j] = i <= nx ? wf[s * (nx + 1) + i] : 0.0;
    }
    const double* Us = U ? U + s * (int64_t)nx * N : nullptr;
    double w[R], v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int i = g * R + j;
        w[j] = i < nx ? ((mode == 1 || n == 0) ? u0[i] : Us[(int64_t)i * N + n - 1]) : 0.0;
    }
    bool ok = true;
    unsigned long long its = 0;
    const double dt = dT / J;
    const int nint = mode == 0 ? 1 : N;
    for (int ni = 0; ni < nint; ++ni) {
        for (int j = 0; j < J; ++j) {
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = w[q];
            ok &= newton_be_g<KIND, G, R>(nx, g, wfv, dt, c, f0, v, w, &its);
        }
        if (mode == 1 && real && act) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int i = g * R + q;
                if (i < nx) out[(s * (int64_t)nx + i) * N + ni] = w[q];
            }
        }
    }
    if (mode == 0 && jump) {
        // G(prev): one step of dT from prev; F stays in w
        double gv[R], gw[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = g * R + q;
            const double pv = i < nx ? (n == 0 ? alpha * Us[(int64_t)i * N + N - 1]
                                               : Us[(int64_t)i * N + n - 1])
                                     : 0.0;
            gv[q] = pv;
            gw[q] = pv;
        }
        ok &= newton_be_g<KIND, G, R>(nx, g, wfv, dT, c, f0, gv, gw, &its);
#pragma unroll
        for (int q = 0; q < R; ++q) w[q] -= gw[q];
    }
    if (mode == 0 && real && act) {
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int i = g * R + q;
            if (i < nx) out[(s * (int64_t)nx + i) * N + n] = w[q];
        }
    }
    if (real && act && g == 0) {
        if (!ok && ifail) ifail[s] = 1;
        if (itcount) atomicAdd(itcount, its);
    }
}

// Lanes per column and rows per lane for nx rows: G = 16 up to 128 rows,
// else 32; R the smallest power of two with G R >= nx, at most 8 (a lane
// holds ~9 R doubles; at R = 16 they spill).  R = 0 past 256 rows: the
// thread-per-column kernel takes those.
void newton_g_shape(int nx, int* G, int* R) {
    *G = nx <= 128 ? 16 : 32;
    *R = 0;
    for (int r : {2, 4, 8})
        if (*G * r >= nx) {
            *R = r;
            break;
        }
}

template <int KIND>
bool launch_newton_g(int64_t S, int N, int nx, int J, double dT, double alpha, double c, double f0,
                     int jump, int mode, const double* U, const double* u0, const double* wf,
                     double* out, const int* active, int* ifail, unsigned long long* itcount,
                     cudaStream_t st) {
    int G = 0, R = 0;
    newton_g_shape(nx, &G, &R);
    if (R == 0) return false;
    const int64_t ncol = mode == 0 ? S * N : S;
    const int64_t threads = ((ncol * G + 31) / 32) * 32;
    const unsigned grid = (unsigned)((threads + 127) / 128);
#define KLECGC_NG(GG, RR)                                                                      \
    if (G == GG && R == RR) {                                                                  \
        k_newton_g<KIND, GG, RR><<<grid, 128, 0, st>>>(S, N, nx, J, dT, alpha, c, f0, jump,    \
                                                        mode, U, u0, wf, out, active, ifail,   \
                                                        itcount);                              \
        return true;                                                                           \
    }
    KLECGC_NG(16, 2)
    KLECGC_NG(16, 4)
    KLECGC_NG(16, 8)
    KLECGC_NG(32, 8)
#undef KLECGC_NG
    return false;
}

}  // namespace

// Host value of the kernels' c: the cubic coefficient (kind 1) or c/h (kind 2).
static double kind_coef(int kind, int nx, double c) { return kind == 2 ? c * (nx + 1) : c; }

void launch_fine_newton(int kind, int64_t S, int N, int nx, int J, double dT, double alpha,
                        double c, double f0, int jump, const double* U, const double* u0,
                        const double* wf, double* b, double* scratch, const int* active,
                        int* ifail, unsigned long long* itcount, cudaStream_t st) {
    const int64_t n = S * N;
    if (n == 0) return;
    const int64_t NS = n * nx;
    const double ck = kind_coef(kind, nx, c);
    // G lanes per column where the rows fit (nx <= 256)
    if (kind == 2 ? launch_newton_g<2>(S, N, nx, J, dT, alpha, ck, f0, jump, 0, U, u0, wf, b,
                                       active, ifail, itcount, st)
                  : launch_newton_g<1>(S, N, nx, J, dT, alpha, ck, f0, jump, 0, U, u0, wf, b,
                                       active, ifail, itcount, st))
        return;
    // One warp per CTA: each thread runs a long dependent FP64 chain, and the
    // FP64 pipe of an SM saturates at a few warps, so a batch of a few
    // thousand columns is spread over all SMs (128-thread CTAs put 256
    // samples x 32 intervals on 64 of the 152 SMs).
    const unsigned grid = (unsigned)((n + 31) / 32);
    if (kind == 2)
        k_fine_newton<2><<<grid, 32, 0, st>>>(S, N, nx, J, dT, alpha, ck, f0, jump, U, u0, wf, b,
                                              scratch, scratch + NS, scratch + 2 * NS,
                                              scratch + 3 * NS, active, ifail, itcount);
    else
        k_fine_newton<1><<<grid, 32, 0, st>>>(S, N, nx, J, dT, alpha, ck, f0, jump, U, u0, wf, b,
                                              scratch, scratch + NS, scratch + 2 * NS,
                                              scratch + 3 * NS, active, ifail, itcount);
}

// Sequential fine solution with Newton steps (reference, snapshots, the
// coarse guess with J = 1): one thread per sample, scratch [4][nx][S].
template <int KIND>
__global__ void __launch_bounds__(64) k_sequential_newton(
    int64_t S, int N, int nx, int J, double dt, double c, double f0, const double* __restrict__ u0,
    const double* __restrict__ wf, double* __restrict__ scr, double* __restrict__ U,
    int* __restrict__ ifail) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int64_t plane = (int64_t)nx * S;
    double* w = scr + s;
    double* v = w + plane;
    double* cp = v + plane;
    double* dp = cp + plane;
    const double* wfs = wf + s * (nx + 1);
    bool ok = true;
    unsigned long long its = 0;
    for (int i = 0; i < nx; ++i) w[(int64_t)i * S] = u0[i];
    double* Us = U + s * (int64_t)nx * N;
    for (int n = 0; n < N; ++n) {
        for (int j = 0; j < J && ok; ++j) {
            for (int i = 0; i < nx; ++i) v[(int64_t)i * S] = w[(int64_t)i * S];
            ok = newton_be<KIND>(nx, wfs, dt, c, f0, v, w, cp, dp, S, &its);
        }
        for (int i = 0; i < nx; ++i) Us[(int64_t)i * N + n] = w[(int64_t)i * S];
    }
    if (!ok && ifail) ifail[s] = 1;
}

void launch_sequential_newton(int kind, int64_t S, int N, int nx, int J, double dt, double c,
                              double f0, const double* u0, const double* wf, double* scratch,
                              double* U, int* ifail, cudaStream_t st) {
    if (S == 0) return;
    const double ck = kind_coef(kind, nx, c);
    if (kind == 2 ? launch_newton_g<2>(S, N, nx, J, dt * J, 0.0, ck, f0, 0, 1, nullptr, u0, wf, U,
                                       nullptr, ifail, nullptr, st)
                  : launch_newton_g<1>(S, N, nx, J, dt * J, 0.0, ck, f0, 0, 1, nullptr, u0, wf, U,
                                       nullptr, ifail, nullptr, st))
        return;
    const unsigned grid = (unsigned)((S + 31) / 32);   // one warp per CTA (see above)
    if (kind == 2)
        k_sequential_newton<2><<<grid, 32, 0, st>>>(S, N, nx, J, dt, ck, f0, u0, wf, scratch, U,
                                                    ifail);
    else
        k_sequential_newton<1><<<grid, 32, 0, st>>>(S, N, nx, J, dt, ck, f0, u0, wf, scratch, U,
                                                    ifail);
}

// Simplified Newton step, part 1: per row (s, i), e_i = c (3 m_i - 1) with
// m_i = mean_n (u_{n,i} - b_{n,i})^2, and
//   rhs_n,i = dT ((A + diag e) u_n)_i + dT f(u_n - b_n)_i + b_n,i.
__global__ void k_nl_prep(int64_t S, int N, int nx, double dT, double c, double f0,
                          const double* __restrict__ u, const double* __restrict__ b,
                          const double* __restrict__ wf, double* __restrict__ rhs,
                          double* __restrict__ e, const int* __restrict__ active) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t s = t / nx;
    const int i = (int)(t - s * nx);
    if (s >= S || !active[s]) return;
    const int64_t row = (s * nx + i) * (int64_t)N;
    const double* ur = u + row;
    const double* br = b + row;
    double m = 0.0;
    for (int n = 0; n < N; ++n) {
        const double z = ur[n] - br[n];
        m = fma(z, z, m);
    }
    const double ei = c * (3.0 * (m / N) - 1.0);
    e[s * nx + i] = ei;
    const double wl = wf[s * (nx + 1) + i], wr = wf[s * (nx + 1) + i + 1];
    const bool hasl = i > 0, hasr = i + 1 < nx;
    for (int n = 0; n < N; ++n) {
        const double ui = ur[n], zi = ui - br[n];
        const double ul = hasl ? ur[n - N] : 0.0, ur_ = hasr ? ur[n + N] : 0.0;
        const double zl = hasl ? ul - br[n - N] : 0.0, zr = hasr ? ur_ - br[n + N] : 0.0;
        const double Au = wl * (ui - ul) - wr * (ur_ - ui);
        const double Az = wl * (zi - zl) - wr * (zr - zi);
        const double fz = -Az - c * (zi * zi * zi - zi) + f0;
        rhs[row + n] = dT * (Au + ei * ui) + dT * fz + br[n];
    }
}

void launch_nl_prep(int64_t S, int N, int nx, double dT, double c, double f0, const double* u,
                    const double* b, const double* wf, double* rhs, double* e, const int* active,
                    cudaStream_t st) {
    const int64_t n = S * nx;
    if (n == 0) return;
    k_nl_prep<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(S, N, nx, dT, c, f0, u, b, wf, rhs, e,
                                                           active);
}

// Simplified Newton step, part 1 for kind 2: per row (s, i) the face
// couplings lo_i, up_i (and lo_nx, up_nx from the last row) of dT K, and
//   rhs_n,i = (dT K u_n)_i + dT f(u_n - b_n)_i + b_n,i.
// ch = c/h.  mean_n max(z, 0) and mean_n min(z, 0) of the rows i-1, i, i+1
// are recomputed by each row's thread (N values each).
__global__ void k_nl_prep_burgers(int64_t S, int N, int nx, double dT, double ch, double f0,
                                  const double* __restrict__ u, const double* __restrict__ b,
                                  const double* __restrict__ wf, double* __restrict__ rhs,
                                  double* __restrict__ lo, double* __restrict__ up,
                                  const int* __restrict__ active) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t s = t / nx;
    const int i = (int)(t - s * nx);
    if (s >= S || !active[s]) return;
    const int64_t row = (s * nx + i) * (int64_t)N;
    double pos[3] = {0.0, 0.0, 0.0}, neg[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < 3; ++d) {
        const int j = i + d - 1;
        if (j < 0 || j >= nx) continue;
        const double* uj = u + row + (int64_t)(d - 1) * N;
        const double* bj = b + row + (int64_t)(d - 1) * N;
        double p = 0.0, m = 0.0;
        for (int n = 0; n < N; ++n) {
            const double z = uj[n] - bj[n];
            p += fmax(z, 0.0);
            m += fmin(z, 0.0);
        }
        pos[d] = p / N;
        neg[d] = m / N;
    }
    const double* wfs = wf + s * (nx + 1);
    const double wl = wfs[i], wr = wfs[i + 1];
    const double lo_i = dT * (wl + ch * pos[0]), up_i = dT * (wl - ch * neg[1]);
    const double lo_r = dT * (wr + ch * pos[1]);
    const double up_r = i + 1 < nx ? dT * (wr - ch * neg[2]) : dT * wr;
    lo[s * (nx + 1) + i] = lo_i;
    up[s * (nx + 1) + i] = up_i;
    if (i + 1 == nx) {
        lo[s * (nx + 1) + nx] = lo_r;
        up[s * (nx + 1) + nx] = up_r;
    }
    const bool hasl = i > 0, hasr = i + 1 < nx;
    const double* ur = u + row;
    const double* br = b + row;
    for (int n = 0; n < N; ++n) {
        const double ui = ur[n], zi = ui - br[n];
        const double ul = hasl ? ur[n - N] : 0.0, uR = hasr ? ur[n + N] : 0.0;
        const double zl = hasl ? ul - br[n - N] : 0.0, zr = hasr ? uR - br[n + N] : 0.0;
        const double Ku = -lo_i * ul + (up_i + lo_r) * ui - up_r * uR;      // (dT K u)_i
        const double Az = wl * (zi - zl) - wr * (zr - zi);
        const double fz = -Az - ch * (eo_flux(zi, zr) - eo_flux(zl, zi)) + f0;
        rhs[row + n] = Ku + dT * fz + br[n];
    }
}

void launch_nl_prep_burgers(int64_t S, int N, int nx, double dT, double c, double f0,
                            const double* u, const double* b, const double* wf, double* rhs,
                            double* lo, double* up, const int* active, cudaStream_t st) {
    const int64_t n = S * nx;
    if (n == 0) return;
    k_nl_prep_burgers<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
        S, N, nx, dT, c * (nx + 1), f0, u, b, wf, rhs, lo, up, active);
}

// Factors of lambda_k I + dT K for a tridiagonal dT K given by its face
// couplings (row i: -lo_i, up_i + lo_{i+1}, -up_{i+1}), one thread per
// (s, k): pivots piv_i = lambda_k + up_i + lo_{i+1} - lo_i up_i / piv_{i-1};
// dinv_i = 1 / piv_i and lu_i = -up_{i+1} / piv_i, the layout k_cgc_solve
// reads (with lo as its lower couplings).
__global__ void k_cgc_factors_faces(int64_t S, int nx, const double* __restrict__ lo,
                                    const double* __restrict__ up,
                                    const double2* __restrict__ lam, int K,
                                    Cplx<double>* __restrict__ dinv, Cplx<double>* __restrict__ lu,
                                    const int* __restrict__ active) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= S * K) return;
    const int64_t s = t / K;
    const int k = (int)(t - s * K);
    if (!active[s]) return;
    const double* los = lo + s * (nx + 1);
    const double* ups = up + s * (nx + 1);
    const double2 lk = lam[k];
    double pr = 1.0, pi = 0.0;
    for (int i = 0; i < nx; ++i) {
        double dr = lk.x + ups[i] + los[i + 1], di = lk.y;
        if (i > 0) {
            const double q = los[i] * ups[i] / (pr * pr + pi * pi);
            dr -= q * pr;
            di += q * pi;
        }
        pr = dr;
        pi = di;
        const double den = pr * pr + pi * pi;
        const double ir = pr / den, ii = -pi / den;
        const int64_t o = (s * nx + i) * K + k;
        dinv[o] = Cplx<double>{ir, ii};
        const double w = i + 1 < nx ? ups[i + 1] : 0.0;
        lu[o] = Cplx<double>{-w * ir, -w * ii};
    }
}

void launch_cgc_factors_faces(int64_t S, int nx, const double* lo, const double* up,
                              const double2* lam, int K, Cplx<double>* dinv, Cplx<double>* lu,
                              const int* active, cudaStream_t st) {
    const int64_t n = S * K;
    if (n == 0) return;
    k_cgc_factors_faces<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(S, nx, lo, up, lam, K, dinv,
                                                                     lu, active);
}

// Classical parareal correction (Algorithm 1, eq. pred_correc) with Newton
// propagators, one thread per sample, in sequence over n:
//     U^{k+1}_n = G(U^{k+1}_{n-1}) + F_n - G(U^k_{n-1}),  U_0 = u0,
// F = F(U^k_{n-1}) the fine end values.  delta[s] = max |U^{k+1} - U^k| (as
// bits).  Scratch [5][nx][S]: G(U^k) iterate, G(U^{k+1}) iterate, start
// value, Thomas c', d'.
template <int KIND>
__global__ void __launch_bounds__(64) k_parareal_correct_newton(
    int64_t S, int N, int nx, double dT, double c, double f0, const double* __restrict__ u0,
    const double* __restrict__ wf, const double* __restrict__ F, double* __restrict__ U,
    double* __restrict__ scr, unsigned long long* __restrict__ delta,
    const int* __restrict__ active, int* __restrict__ ifail) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= S || !active[s]) return;
    const int64_t plane = (int64_t)nx * S;
    double* gold = scr + s;
    double* vnew = gold + plane;
    double* v = vnew + plane;
    double* cp = v + plane;
    double* dp = cp + plane;
    const double* wfs = wf + s * (nx + 1);
    const double* Fs = F + s * (int64_t)nx * N;
    double* Us = U + s * (int64_t)nx * N;
    unsigned long long its = 0;
    bool ok = true;
    for (int i = 0; i < nx; ++i) {
        gold[(int64_t)i * S] = u0[i];
        vnew[(int64_t)i * S] = u0[i];
        v[(int64_t)i * S] = u0[i];
    }
    ok = newton_be<KIND>(nx, wfs, dT, c, f0, v, gold, cp, dp, S, &its);   // G(U^k_0)
    double dmax = 0.0;
    bool bad = false;
    for (int n = 0; n < N; ++n) {
        for (int i = 0; i < nx; ++i) v[(int64_t)i * S] = vnew[(int64_t)i * S];
        if (ok) ok = newton_be<KIND>(nx, wfs, dT, c, f0, v, vnew, cp, dp, S, &its);
        for (int i = 0; i < nx; ++i) {
            const int64_t o = (int64_t)i * N + n;
            const double uold = Us[o];
            const double unew = vnew[(int64_t)i * S] + Fs[o] - gold[(int64_t)i * S];
            gold[(int64_t)i * S] = uold;   // start of G(U^k_n) for the next n
            vnew[(int64_t)i * S] = unew;
            Us[o] = unew;
            const double d = fabs(unew - uold);
            dmax = fmax(dmax, d);
            bad |= d != d;
        }
        if (n + 1 < N) {
            for (int i = 0; i < nx; ++i) v[(int64_t)i * S] = gold[(int64_t)i * S];
            if (ok) ok = newton_be<KIND>(nx, wfs, dT, c, f0, v, gold, cp, dp, S, &its);
        }
    }
    if (!ok) ifail[s] = 1;
    delta[s] = bad ? 0x7ff8000000000000ull : (unsigned long long)__double_as_longlong(dmax);
}

void launch_parareal_correct_newton(int kind, int64_t S, int N, int nx, double dT, double c,
                                    double f0, const double* u0, const double* wf,
                                    const double* F, double* U, double* scratch,
                                    unsigned long long* delta, const int* active, int* ifail,
                                    cudaStream_t st) {
    if (S == 0) return;
    const double ck = kind_coef(kind, nx, c);
    const unsigned grid = (unsigned)((S + 31) / 32);   // one warp per CTA (see above)
    if (kind == 2)
        k_parareal_correct_newton<2><<<grid, 32, 0, st>>>(S, N, nx, dT, ck, f0, u0, wf, F, U,
                                                          scratch, delta, active, ifail);
    else
        k_parareal_correct_newton<1><<<grid, 32, 0, st>>>(S, N, nx, dT, ck, f0, u0, wf, F, U,
                                                          scratch, delta, active, ifail);
}

}  // namespace klecgc
