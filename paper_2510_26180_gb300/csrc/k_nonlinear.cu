// Nonlinear 1D problem (Allen-Cahn-type reaction) and the nonlinear coarse
// grid correction by simplified Newton (Section 3.2, eqs. Newton, Jac, Newton2).
//
//   f(u) = -A u - c (u^3 - u) + f0,   grad f(u) = -A - c diag(3 u^2 - 1),
// A the flux-form operator with face weights wf_i = a_{i-1/2} / h^2.
//
// Backward Euler (both propagators): one step of size dt solves
//     w + dt A w + dt c (w^3 - w) = v + dt f0
// by Newton's method from w = v: the Jacobian I + dt A + dt c diag(3 w^2 - 1) is
// tridiagonal and factored anew in every Newton iteration (Thomas), stopping
// when max |dw| <= 1e-14 max(1, max |w|) (at most kNewtonMax iterations; a step
// that reaches the cap sets the sample's flag).
//
// CGC: eq. matrix_NT, (C_alpha (x) I) u = dT F(u) + b, F(u)_n = f(U_n - b_n), by
// simplified Newton steps from u_0 = U^k:
//     Jbar u_{l+1} = dT (I (x) K) u_l + dT F(u_l) + b,  K = -gradf_bar = A + diag(e),
//     e_i = c (3 m_i - 1),  m_i = (1/N) sum_n (U_{n,i} - b_{n,i})^2   (eq. Jac),
// Jbar = C_alpha (x) I + dT I (x) K: the linear three steps with the shifted
// factors built from the diagonal extra dT e (k_nl_prep writes e and the
// right-hand side; the transforms and solves are the linear kernels).
//
// Layout: U, b, rhs [S][nx][N]; columns (s, n) are strided by N (a warp of
// consecutive n coalesces).
#include "common.cuh"

namespace klecgc {

namespace {

constexpr int kNewtonMax = 50;

// One Newton backward-Euler step on the column w (stride st): v is the start
// value (overwritten by nothing), w the iterate (in/out), cp / dp Thomas
// scratch.  wf: face weights a/h^2 (nx + 1), dt, c, f0.  Returns false if the
// iteration cap was reached; adds the Newton iterations taken to *its.
__device__ bool newton_be(int nx, const double* __restrict__ wf, double dt, double c,
                          double f0, const double* v, double* w, double* cp, double* dp,
                          int64_t st, unsigned long long* its) {
    for (int it = 0; it < kNewtonMax; ++it) {
        ++*its;
        // residual R = w + dt A w + dt c (w^3 - w) - v - dt f0 and the Thomas
        // forward elimination of (I + dt A + dt c diag(3 w^2 - 1)) d = R
        double wl = 0.0, wi = w[0], prevc = 0.0, prevd = 0.0;
        for (int i = 0; i < nx; ++i) {
            const double wr = i + 1 < nx ? w[(int64_t)(i + 1) * st] : 0.0;
            const double fl = dt * wf[i], fr = dt * wf[i + 1];
            const double Aw = fl * (wi - wl) - fr * (wr - wi);          // dt A w
            const double R = wi + Aw + dt * c * (wi * wi * wi - wi) - v[(int64_t)i * st] - dt * f0;
            const double diag = 1.0 + fl + fr + dt * c * (3.0 * wi * wi - 1.0);
            // row i: -fl d_{i-1} + diag d_i - fr d_{i+1} = R
            const double den = diag + fl * prevc;                    // diag - (-fl) c'_{i-1}
            const double ci = -fr / den;                             // c'_i (upper / pivot)
            const double di = (R + fl * prevd) / den;
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

// F (J steps of dt = dT/J from start_n = u0 or U_{n-1}) and the jump
// b_n = F_n - G(prev_n), prev_1 = alpha U_N, prev_n = U_{n-1}, per column (s, n).
// Scratch: v, cp, dp, g [S][nx][N]; bout receives b (and holds F meanwhile).
__global__ void __launch_bounds__(128) k_fine_newton(
    int64_t S, int N, int nx, int J, double dT, double alpha, double c, double f0,
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
        ok = newton_be(nx, wfs, dt, c, f0, v, w, cp, dp, N, &its);
    }
    // G(prev): one step of dT from prev (start v, iterate g); F stays in w
    double* g = gs + base;
    for (int i = 0; i < nx; ++i) {
        const double pv = n == 0 ? alpha * Us[(int64_t)i * N + N - 1] : Us[(int64_t)i * N + n - 1];
        v[(int64_t)i * N] = pv;
        g[(int64_t)i * N] = pv;
    }
    if (ok) ok = newton_be(nx, wfs, dT, c, f0, v, g, cp, dp, N, &its);
    for (int i = 0; i < nx; ++i) w[(int64_t)i * N] -= g[(int64_t)i * N];
    if (!ok) ifail[s] = 1;
    if (itcount) atomicAdd(itcount, its);
}

void launch_fine_newton(int64_t S, int N, int nx, int J, double dT, double alpha, double c,
                        double f0, const double* U, const double* u0, const double* wf, double* b,
                        double* scratch, const int* active, int* ifail,
                        unsigned long long* itcount, cudaStream_t st) {
    const int64_t n = S * N;
    if (n == 0) return;
    const int64_t NS = n * nx;
    k_fine_newton<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
        S, N, nx, J, dT, alpha, c, f0, U, u0, wf, b, scratch, scratch + NS, scratch + 2 * NS,
        scratch + 3 * NS, active, ifail, itcount);
}

// Sequential fine solution with Newton steps (reference, snapshots, the
// coarse guess with J = 1): one thread per sample, scratch [4][nx][S].
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
            ok = newton_be(nx, wfs, dt, c, f0, v, w, cp, dp, S, &its);
        }
        for (int i = 0; i < nx; ++i) Us[(int64_t)i * N + n] = w[(int64_t)i * S];
    }
    if (!ok && ifail) ifail[s] = 1;
}

void launch_sequential_newton(int64_t S, int N, int nx, int J, double dt, double c, double f0,
                              const double* u0, const double* wf, double* scratch, double* U,
                              int* ifail, cudaStream_t st) {
    if (S == 0) return;
    k_sequential_newton<<<(unsigned)((S + 63) / 64), 64, 0, st>>>(S, N, nx, J, dt, c, f0, u0, wf,
                                                                  scratch, U, ifail);
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

}  // namespace klecgc
