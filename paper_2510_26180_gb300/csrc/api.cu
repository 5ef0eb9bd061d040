// C ABI of libklecgc: context, setup (offline part of Algorithm 3) and the
// solve loop (online part: Algorithm 2 from the surrogate guess).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/klecgc.h"
#include "common.cuh"
#include "setup_host.h"

namespace klecgc {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// Learned-guess network M -> W -> W -> W -> D (D = 64 N), flat FP32 parameters
// [W1, b1, W2, b2, W3, b3, W4, b4] with W_l stored [out][in].
struct MlpState {
    int sizes[5] = {0, 0, 0, 0, 0};
    int64_t woff[4] = {0, 0, 0, 0}, boff[4] = {0, 0, 0, 0};
    int64_t P = 0;
    int D = 0;
    float* theta = nullptr;      // FP32 master parameters
    __nv_bfloat16* thb = nullptr;  // BF16 copy (GEMM operands)
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* mean = nullptr;       // [D] output normalization
    float* stdv = nullptr;
    float* inv_std = nullptr;
    int adam_t = 0;
    bool ready = false;
    bool residual = false;       // output is a correction added to the gPC guess
};

}  // namespace klecgc

using namespace klecgc;

struct klecgc_ctx {
    klecgc_problem prob{};
    int device = 0;
    int nx = 0, N = 0, J = 0, M = 0, P = 0, MQ = 0, p = 0;
    int dim = 1;
    int ns = 0;   // unknowns nx^dim
    int nf = 0;   // coefficient faces per sample: nx+1 (1D), 2 nx (nx+1) (2D)
    // 2D Krylov solves: relative residual tolerances, iteration cap, counters
    double kry_rtol_fine = 1e-10, kry_rtol_cgc = 1e-10;
    int kry_maxit = 10000;
    unsigned long long kry_it_fine = 0, kry_it_cgc = 0;
    double h = 0.0, dT = 0.0;
    double lambda_sum = 0.0, lambda_kept = 0.0;
    // device tables (owned)
    double* basis = nullptr;   // [M][nf]  sqrt(lambda_m) phi_m at the faces
    double* u0 = nullptr;      // [ns]
    int* degrees = nullptr;    // [P][M]
    double* ubar = nullptr;    // [ns*N]  internal order c = i*N + n
    float2* ubar_df = nullptr; // the same as FP32 pairs (hi, lo) (guess in pair format)
    double* W = nullptr;       // [P][ns*N]
    float* W32 = nullptr;      // FP32 copy of W
    float* W32t = nullptr;     // [ns*N][Kp] TF32 head of W^T, zero-padded (tensor-core guess)
    float* W32t_lo = nullptr;  // [ns*N][Kp] its tail W^T - head
    int Kp = 0;
    int* tc_err = nullptr;     // set by the tensor-core guess when a wait timed out
    int method2d = 0;          // 2D linear solves: 0 auto, 1 Krylov, 2 banded LU, 3 Krylov on clusters
    int loop_mode = 0;         // parareal loop: 0 CUDA graph (WHILE node), 1 host-driven
    // launch-shape autotuner: 1 times the candidate shapes once per problem
    // shape (and GPU) and keeps the fastest; 0 uses the fixed rules
    int tune_mode = 1;
    std::map<std::string, std::string> tuned;   // key -> chosen shape
    std::string tune_path;                      // JSON cache file ("" = none)
    std::string gpu_name;                       // the device's name (tuner keys), read once
    bool fine_smem_only = false;                // the batch's persistent fine stage runs k_fine32
    bool mlp_tc = true;                         // network GEMMs on tcgen05 where the shape allows
    std::map<std::string, DevBuf> ws;  // grow-only scratch
    size_t ws_limit = 0;               // bytes of scratch allowed (0: no limit)
    std::string ws_tag;                // appended to scratch names (one batch class each)
    std::vector<void*> owned;
    MlpState mlp;
    // profile: launch counters and optional CUDA-event timing per kernel class
    bool prof_timing = false;
    int64_t prof_launches[KLECGC_K_COUNT] = {};
    double prof_ms[KLECGC_K_COUNT] = {};
    std::vector<cudaEvent_t> prof_free;
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Pending> prof_pending;

    cudaEvent_t prof_event() {
        if (!prof_free.empty()) {
            cudaEvent_t e = prof_free.back();
            prof_free.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    // Runs `f` (one kernel launch) under class `cls`.
    template <class F>
    void launch(int cls, cudaStream_t st, F&& f) {
        prof_launches[cls] += 1;
        if (!prof_timing) {
            f();
            return;
        }
        cudaEvent_t a = prof_event(), b = prof_event();
        cudaEventRecord(a, st);
        f();
        cudaEventRecord(b, st);
        prof_pending.push_back({cls, a, b});
    }
    void prof_collect() {
        for (auto& p : prof_pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
                prof_ms[p.cls] += ms;
            prof_free.push_back(p.a);
            prof_free.push_back(p.b);
        }
        prof_pending.clear();
    }

    template <typename T>
    T* get(const std::string& name, size_t count, cudaError_t* err) {
        DevBuf& b = ws[ws_tag.empty() ? name : name + ws_tag];
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (b.bytes < bytes) {
            if (ws_limit) {
                // the caller's budget for the scratch: the sum after growing this buffer
                size_t total = 0;
                for (auto& kv : ws) total += kv.second.bytes;
                if (total - b.bytes + bytes > ws_limit) {
                    *err = cudaErrorMemoryAllocation;
                    return nullptr;
                }
            }
            if (b.ptr) cudaFree(b.ptr);
            b.ptr = nullptr;
            b.bytes = 0;
            cudaError_t e = cudaMalloc(&b.ptr, bytes);
            if (e != cudaSuccess) {
                *err = e;
                return nullptr;
            }
            b.bytes = bytes;
        }
        return (T*)b.ptr;
    }
    template <typename T>
    cudaError_t alloc_owned(T** p, size_t count) {
        cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    }
    ~klecgc_ctx() {
        prof_collect();
        for (cudaEvent_t e : prof_free) cudaEventDestroy(e);
        for (void* p : owned) cudaFree(p);
        for (auto& kv : ws)
            if (kv.second.ptr) cudaFree(kv.second.ptr);
    }
};

namespace klecgc {
bool ctx_view(const klecgc_ctx* ctx, CtxView* out) {
    if (!ctx || !ctx->basis) return false;
    *out = CtxView{ctx->basis, ctx->u0, ctx->nx, ctx->M, ctx->device,
                   ctx->h, ctx->prob.T, ctx->prob.reaction, ctx->prob.forcing, ctx->dim,
                   ctx->prob.reaction_kind};
    return true;
}
}  // namespace klecgc

namespace {

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

klecgc_status fail(klecgc_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

#define TRY(expr)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? KLECGC_E_OUT_OF_MEMORY          \
                                                        : KLECGC_E_CUDA,                \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define WS(T, var, name, count)                                      \
    cudaError_t var##_e = cudaSuccess;                               \
    T* var = ctx->get<T>(name, (size_t)(count), &var##_e);           \
    if (!var) TRY(var##_e)

// Stage a caller array on the device: returns a device pointer holding the data.
template <typename T>
klecgc_status stage_in(klecgc_ctx* ctx, const T* user, size_t count, const char* name,
                       cudaStream_t st, const T** out) {
    if (is_device_ptr(user)) {
        *out = user;
        return KLECGC_OK;
    }
    WS(T, d, name, count);
    TRY(cudaMemcpyAsync(d, user, count * sizeof(T), cudaMemcpyHostToDevice, st));
    *out = d;
    return KLECGC_OK;
}

bool pow2_in_range(int N) { return N >= 2 && N <= 64 && (N & (N - 1)) == 0; }

// Relative tolerance of the FP32 inner solves of the mixed 2D propagator (each
// FP64 refinement gains about this factor).
constexpr double kInnerRtol = 1e-4;

klecgc_status check_dT(const klecgc_ctx* ctx, int N, double dT) {
    double T = ctx->prob.T;
    if (!(dT > 0) || std::fabs(N * dT - T) > 1e-12 * T)
        return fail(KLECGC_E_INVALID_ARG, "N * dT must equal T");
    return KLECGC_OK;
}

// Per-solve operators: coefficient field, face weights, fine and CGC factors.
struct Operators {
    double* a = nullptr;
    double* wT = nullptr;
    FineCoef64* f64 = nullptr;
    FineCoef32* f32 = nullptr;
    float* tab32 = nullptr;
    Fine32wShape sh32{0, 0};
    Cplx<double>* dinv64 = nullptr;
    Cplx<double>* lu64 = nullptr;
    Cplx<float>* dinv32 = nullptr;
    Cplx<float>* lu32 = nullptr;
    float* wT32 = nullptr;
};

klecgc_status build_field(klecgc_ctx* ctx, const double* xi_d, int64_t S, cudaStream_t st,
                          double** a_out) {
    const int nf = ctx->nf;
    WS(double, a, "a", S * nf);
    ctx->launch(KLECGC_K_FIELD, st, [&] { launch_field(xi_d, S, ctx->M, ctx->basis, nf, a, st); });
    TRY(cudaGetLastError());
    *a_out = a;
    return KLECGC_OK;
}

// Eigenvalues lambda_k = 1 - alpha^{1/N} exp(-2 pi i k / N), k = 0..N/2, of
// C_alpha (host copy in lam, device copy in *lam_d).
klecgc_status upload_lambda(klecgc_ctx* ctx, int N, double alpha, cudaStream_t st,
                            std::vector<double2>& lam, double2** lam_d) {
    const int K = N / 2 + 1;
    lam.resize(K);
    const double a1n = std::pow(alpha, 1.0 / N), pi = 3.14159265358979323846;
    for (int k = 0; k < K; ++k) {
        lam[k].x = 1.0 - a1n * std::cos(2.0 * pi * k / N);
        lam[k].y = a1n * std::sin(2.0 * pi * k / N);
    }
    WS(double2, d, "lam", K);
    TRY(cudaMemcpyAsync(d, lam.data(), K * sizeof(double2), cudaMemcpyHostToDevice, st));
    *lam_d = d;
    return KLECGC_OK;
}

// want_fine: 0 none, 1 FP64, 2 FP64+FP32; want_cgc: 0 none, 1 FP64, 2 FP32.
// ---- launch-shape autotuner
// Keys are "<GPU name>|<kernel>|nx=..|N=..|J=.."; values the chosen shape.
// The cache file is a flat JSON object of such strings.
std::string tune_key(klecgc_ctx* ctx, const char* kernel, int nx, int N, int J) {
    if (ctx->gpu_name.empty()) {
        cudaDeviceProp prop;
        ctx->gpu_name = cudaGetDeviceProperties(&prop, ctx->device) == cudaSuccess ? prop.name : "?";
    }
    return ctx->gpu_name + "|" + kernel + "|nx=" + std::to_string(nx) + "|N=" +
           std::to_string(N) + "|J=" + std::to_string(J);
}

std::string tune_json(const klecgc_ctx* ctx) {
    std::string out = "{";
    bool first = true;
    for (auto& kv : ctx->tuned) {
        out += first ? "\n" : ",\n";
        out += "  \"" + kv.first + "\": \"" + kv.second + "\"";
        first = false;
    }
    return out + (first ? "}" : "\n}");
}

// Reads "key": "value" pairs of a flat JSON object (the format tune_json
// writes) into the choices.
void tune_parse(klecgc_ctx* ctx, const std::string& txt) {
    size_t pos = 0;
    std::vector<std::string> strs;
    while ((pos = txt.find('"', pos)) != std::string::npos) {
        const size_t end = txt.find('"', pos + 1);
        if (end == std::string::npos) break;
        strs.push_back(txt.substr(pos + 1, end - pos - 1));
        pos = end + 1;
    }
    for (size_t i = 0; i + 1 < strs.size(); i += 2) ctx->tuned[strs[i]] = strs[i + 1];
}

void tune_load(klecgc_ctx* ctx) {
    if (ctx->tune_path.empty()) return;
    FILE* f = std::fopen(ctx->tune_path.c_str(), "rb");
    if (!f) return;
    std::string txt;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, n);
    std::fclose(f);
    tune_parse(ctx, txt);
}

void tune_save(const klecgc_ctx* ctx) {
    if (ctx->tune_path.empty()) return;
    FILE* f = std::fopen(ctx->tune_path.c_str(), "wb");
    if (!f) return;
    const std::string j = tune_json(ctx);
    std::fwrite(j.data(), 1, j.size(), f);
    std::fclose(f);
}

// Launch shape of the FP32 fine propagator for (nx, N, J): with tuning on,
// the first call for a shape times every candidate (W warps per pair of
// intervals, R rows per lane) on up to 512 samples of this solve (F0 of zero
// increments, in_mode 1: the work does not depend on the values) and keeps
// the fastest; afterwards, and with tuning off, it is a lookup or the rule.
klecgc_status choose_fine32w(klecgc_ctx* ctx, int64_t S, int N, int nx, int J, double dt,
                             const double* a, const FineCoef64* f64, cudaStream_t st,
                             Fine32wShape* out) {
    // candidate W = 0: k_fine32 (one warp per pair of intervals, the factors
    // in shared memory, R rows per lane by its own rule); W >= 1: k_fine32w;
    // L >= 1: k_fine32r (one interval per warp, factors in registers, L
    // intervals per warp in turn); P: k_fine32p (one interval per warp, each
    // lane's rows as two halves in packed FP32x2)
    const int R0 = fine32_rows_per_lane(nx);
    *out = {0, R0};
    std::vector<Fine32wShape> cands;
    if (R0) cands.push_back({0, R0});
    if (!ctx->fine_smem_only) {
        for (const Fine32wShape& c : fine32w_candidates(nx)) cands.push_back(c);
        for (int L : {1, 4})
            if (fine32r_supported(R0, L)) cands.push_back({0, R0, L});
        if (fine32p_supported(R0)) cands.push_back({0, R0, 0, 1});
    }
    if (ctx->tune_mode == 0 || cands.size() < 2 || S == 0) return KLECGC_OK;
    const std::string key = tune_key(ctx, "fine32", nx, N, J);
    auto decode = [&](const std::string& v, Fine32wShape* sh) {
        int W = 0, R = 0;
        if (std::sscanf(v.c_str(), "W%dR%d", &W, &R) == 2) {
            *sh = {W, R};
            return W == 0 ? R == R0 : fine32w_supported(*sh);
        }
        if (std::sscanf(v.c_str(), "L%dR%d", &W, &R) == 2) {
            *sh = {0, R, W};
            return R == R0 && fine32r_supported(R, W);
        }
        if (std::sscanf(v.c_str(), "P%dR%d", &W, &R) == 2) {
            *sh = {0, R, 0, 1};
            return W == 1 && R == R0 && fine32p_supported(R);
        }
        return false;
    };
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end() && decode(it->second, out)) return KLECGC_OK;
    const int64_t St = std::min<int64_t>(S, 512);
    size_t tab = R0 ? fine_table32_bytes(St, R0) : 0;
    for (auto& c : cands) {
        if (c.P) tab = std::max(tab, fine_table32p_bytes(St, c.R));
        else if (c.L) tab = std::max(tab, fine_table32r_bytes(St, c.R));
        else if (c.W) tab = std::max(tab, fine_table32w_bytes(St, c));
    }
    WS(float, tb, "tune_table", tab / sizeof(float));
    WS(float, cz, "tune_c", St * (int64_t)nx * N);
    WS(float, fo, "tune_out", St * (int64_t)nx * N);
    WS(int, act, "tune_active", St);
    TRY(cudaMemsetAsync(cz, 0, St * (int64_t)nx * N * sizeof(float), st));
    TRY(cudaMemsetAsync(act, 0xff, St * sizeof(int), st));
    cudaEvent_t e0, e1;
    TRY(cudaEventCreate(&e0));
    TRY(cudaEventCreate(&e1));
    float best = 0.f;
    Fine32wShape pick = *out;
    auto name = [](const Fine32wShape& c) {
        return c.P   ? "P1R" + std::to_string(c.R)
               : c.L ? "L" + std::to_string(c.L) + "R" + std::to_string(c.R)
                     : "W" + std::to_string(c.W) + "R" + std::to_string(c.R);
    };
    std::string times;
    auto run = [&](const Fine32wShape& c) {
        launch_fine_any(c, St, N, nx, J, dt, 0.0, 0.0, 1, nullptr, nullptr, ctx->u0, cz, tb, fo,
                        act, st);
    };
    for (const Fine32wShape& c : cands) {
        if (c.P)
            launch_fine_table32p(f64, St, nx, c.R, tb, st);
        else if (c.L)
            launch_fine_table32r(f64, St, nx, c.R, tb, st);
        else if (c.W == 0)
            launch_fine_table32(a, St, nx, c.R, ctx->h, dt, ctx->prob.reaction, tb, st);
        else
            launch_fine_table32w(f64, St, nx, c, tb, st);
        run(c);   // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2; ++r) run(c);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(KLECGC_E_CUDA, std::string("autotuner: ") + cudaGetErrorString(e));
        }
        if (best == 0.f || ms < best) {
            best = ms;
            pick = c;
        }
        char buf[48];
        std::snprintf(buf, sizeof(buf), "%s%s:%.4f", times.empty() ? "" : " ", name(c).c_str(),
                      ms / 2);
        times += buf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TRY(cudaGetLastError());
    *out = pick;
    ctx->tuned[key] = name(pick);
    // the measured candidates (ms per launch on St samples), for the record
    ctx->tuned[key + "|ms@S=" + std::to_string(St)] = times;
    tune_save(ctx);
    return KLECGC_OK;
}

klecgc_status build_operators(klecgc_ctx* ctx, const double* xi_d, int64_t S, int N, int J,
                              double dT, double alpha, int want_fine, int want_cgc,
                              cudaStream_t st, Operators* op) {
    const int nx = ctx->nx, nf = nx + 1, K = N / 2 + 1;
    klecgc_status s = build_field(ctx, xi_d, S, st, &op->a);
    if (s != KLECGC_OK) return s;
    {
        WS(double, wT, "wT", S * nf);
        ctx->launch(KLECGC_K_FIELD, st, [&] { launch_face_weights(op->a, S, nf, dT / (ctx->h * ctx->h), wT, st); });
        op->wT = wT;
    }
    if (want_fine == 1) {
        WS(FineCoef64, f64, "fine64", S * nf);
        ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_factors(op->a, S, nx, ctx->h, dT / J, ctx->prob.reaction, f64, nullptr, st); });
        op->f64 = f64;
    } else if (want_fine == 2) {
        // FP32 fine propagator: its factors in FP32, in the layout of the
        // kernel and launch shape the autotuner (or the rule) picks
        if (!fine32_rows_per_lane(nx))
            return fail(KLECGC_E_UNSUPPORTED, "mixed precision needs nx <= 2047");
        WS(FineCoef64, f64, "fine64", S * nf);
        ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_factors(op->a, S, nx, ctx->h, dT / J, ctx->prob.reaction, f64, nullptr, st); });
        Fine32wShape sh;
        if ((s = choose_fine32w(ctx, S, N, nx, J, dT / J, op->a, f64, st, &sh)) != KLECGC_OK)
            return s;
        const size_t tbytes = sh.P   ? fine_table32p_bytes(S, sh.R)
                              : sh.L ? fine_table32r_bytes(S, sh.R)
                              : sh.W ? fine_table32w_bytes(S, sh)
                                     : fine_table32_bytes(S, sh.R);
        WS(float, tb, "tab32w", tbytes / sizeof(float));
        if (sh.P)
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_table32p(f64, S, nx, sh.R, tb, st); });
        else if (sh.L)
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_table32r(f64, S, nx, sh.R, tb, st); });
        else if (sh.W)
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_table32w(f64, S, nx, sh, tb, st); });
        else
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_table32(op->a, S, nx, sh.R, ctx->h, dT / J, ctx->prob.reaction, tb, st); });
        op->tab32 = tb;
        op->sh32 = sh;
    }
    if (want_cgc) {
        std::vector<double2> lam;
        double2* lam_d = nullptr;
        klecgc_status ls = upload_lambda(ctx, N, alpha, st, lam, &lam_d);
        if (ls != KLECGC_OK) return ls;
        if (want_cgc == 1) {
            WS(Cplx<double>, di, "cgc_dinv64", S * nx * K);
            WS(Cplx<double>, lu, "cgc_lu64", S * nx * K);
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_cgc_factors<double>(op->a, S, nx, ctx->h, dT, ctx->prob.reaction, lam_d, K, di, lu, st); });
            op->dinv64 = di;
            op->lu64 = lu;
        } else {
            std::vector<float2> lam32(K);
            for (int k = 0; k < K; ++k) lam32[k] = make_float2((float)lam[k].x, (float)lam[k].y);
            WS(float2, lam32_d, "lam32", K);
            TRY(cudaMemcpyAsync(lam32_d, lam32.data(), K * sizeof(float2), cudaMemcpyHostToDevice, st));
            WS(float, wT32, "wT32", S * nf);
            WS(Cplx<float>, di, "cgc_dinv32", S * nx * K);
            WS(Cplx<float>, lu, "cgc_lu32", S * nx * K);
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_to_float(op->wT, wT32, S * nf, st); });
            ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_cgc_factors32(wT32, S, nx, dT * ctx->prob.reaction, lam32_d, K, di, lu, st); });
            op->dinv32 = di;
            op->lu32 = lu;
            op->wT32 = wT32;
        }
    }
    TRY(cudaGetLastError());
    return KLECGC_OK;
}

// 2D: coefficient field and the face weights dt a / h^2 (fine, if wdt) and
// dT a / h^2 (CGC, if wdT), layout [S][nf].
klecgc_status build_weights_2d(klecgc_ctx* ctx, const double* xi_d, int64_t S, double dt,
                               double dT, cudaStream_t st, double** wdt, double** wdT) {
    const int nf = ctx->nf;
    double* a = nullptr;
    klecgc_status s = build_field(ctx, xi_d, S, st, &a);
    if (s != KLECGC_OK) return s;
    const double ih2 = 1.0 / (ctx->h * ctx->h);
    if (wdt) {
        WS(double, w, "w2d_fine", S * nf);
        ctx->launch(KLECGC_K_FIELD, st, [&] { launch_face_weights(a, S, nf, dt * ih2, w, st); });
        *wdt = w;
    }
    if (wdT) {
        WS(double, w, "w2d_cgc", S * nf);
        ctx->launch(KLECGC_K_FIELD, st, [&] { launch_face_weights(a, S, nf, dT * ih2, w, st); });
        *wdT = w;
    }
    TRY(cudaGetLastError());
    return KLECGC_OK;
}

// Per-sample flags of Krylov solves that reached the iteration cap, and the
// iteration counter, zeroed.
klecgc_status krylov_flags(klecgc_ctx* ctx, int64_t S, cudaStream_t st, int** ifail,
                           unsigned long long** its) {
    WS(int, f, "kry_fail", S);
    WS(unsigned long long, c, "kry_its", 2);
    TRY(cudaMemsetAsync(f, 0, S * sizeof(int), st));
    TRY(cudaMemsetAsync(c, 0, 2 * sizeof(unsigned long long), st));
    *ifail = f;
    *its = c;
    return KLECGC_OK;
}

// Reads the counters of krylov_flags after the stream work; true if some
// sample's solve reached the cap (its samples are listed in ifail).
klecgc_status krylov_read(klecgc_ctx* ctx, int64_t S, const int* ifail,
                          const unsigned long long* its, cudaStream_t st, std::vector<int>* hf,
                          bool* any) {
    unsigned long long h[2] = {0, 0};
    hf->assign(S, 0);
    TRY(cudaMemcpyAsync(h, its, sizeof(h), cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hf->data(), ifail, S * sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    ctx->kry_it_fine = h[0];
    ctx->kry_it_cgc = h[1];
    *any = false;
    for (int v : *hf) *any |= v != 0;
    return KLECGC_OK;
}

constexpr int kBandMaxNx = 64;    // largest grid the banded LU accepts
constexpr int kBandAutoNx = 32;   // largest grid it is chosen for by default

// 2D FP64 linear solves by banded LU (one factorization per solve, one
// substitution per step) instead of Krylov iterations: by default on grids
// up to kBandAutoNx (above it the factors, nx^3 values per matrix, are
// streamed from memory in every step by too few threads to pay off; at
// nx = 63 with 64 samples the banded path measured 2.8x slower than FP64
// Krylov),
// or as the context forces.
bool use_band(const klecgc_ctx* ctx, bool fp64) {
    if (ctx->dim != 2 || !fp64 || ctx->method2d == 1 || ctx->method2d == 3) return false;
    return ctx->method2d == 2 || ctx->nx <= kBandAutoNx;
}

// Factors of I + step (A + cI) + convection from step-weighted faces w.
klecgc_status band_factors_fine(klecgc_ctx* ctx, const double* w, int64_t S, double step,
                                cudaStream_t st, double** Bf_out) {
    WS(double, Bf, "band_fine", S * band_doubles(ctx->nx));
    ctx->launch(KLECGC_K_FACTORS, st, [&] {
        launch_band_factor_fine(S, ctx->nx, w, step * ctx->prob.reaction,
                                step * ctx->prob.advection, Bf, st);
    });
    TRY(cudaGetLastError());
    *Bf_out = Bf;
    return KLECGC_OK;
}

// Factors of lambda_k I + dT (A + cI) + convection, k = 0..K-1.
klecgc_status band_factors_cgc(klecgc_ctx* ctx, const double* wdT, int64_t S, int K, double dT,
                               const double2* lam_d, cudaStream_t st, double2** Bc_out) {
    WS(double2, Bc, "band_cgc", S * K * band_doubles(ctx->nx));
    ctx->launch(KLECGC_K_FACTORS, st, [&] {
        launch_band_factor_cgc(S, K, ctx->nx, wdT, dT * ctx->prob.reaction,
                               dT * ctx->prob.advection, lam_d, Bc, st);
    });
    TRY(cudaGetLastError());
    *Bc_out = Bc;
    return KLECGC_OK;
}

// 2D plan kinds: BiCGStab with advection, else CG / COCG (or their mixed forms).
int fine_kind(const klecgc_ctx* ctx, bool mixed) {
    return ctx->prob.advection > 0 ? 4 : (mixed ? 2 : 0);
}
int cgc_kind(const klecgc_ctx* ctx, bool mixed) {
    return ctx->prob.advection > 0 ? 5 : (mixed ? 3 : 1);
}

// Sequential fine solution of the 2D problem: out [S][ns][N] (internal layout).
klecgc_status sequential_2d(klecgc_ctx* ctx, const double* xi_d, int64_t S, int N, int J,
                            double* out, cudaStream_t st, bool* capped) {
    const double dT = ctx->prob.T / N, dt = dT / J;
    double* wdt = nullptr;
    klecgc_status s = build_weights_2d(ctx, xi_d, S, dt, dT, st, &wdt, nullptr);
    if (s != KLECGC_OK) return s;
    if (use_band(ctx, true)) {
        double* Bf = nullptr;
        if ((s = band_factors_fine(ctx, wdt, S, dt, st, &Bf)) != KLECGC_OK) return s;
        WS(int, act, "act_all", S);
        WS(double, xs, "band_x", S * (int64_t)ctx->ns);
        TRY(cudaMemsetAsync(act, 0xff, S * sizeof(int), st));
        ctx->launch(KLECGC_K_FINE, st, [&] {
            launch_band_fine(S, N, ctx->nx, J, dt * ctx->prob.reaction, dt * ctx->prob.forcing,
                             dt * ctx->prob.advection, 0.0, 1, nullptr, ctx->u0, wdt, Bf, xs, out,
                             act, st);
        });
        TRY(cudaGetLastError());
        ctx->kry_it_fine = ctx->kry_it_cgc = 0;
        *capped = false;
        return KLECGC_OK;
    }
    int* ifail = nullptr;
    unsigned long long* its = nullptr;
    if ((s = krylov_flags(ctx, S, st, &ifail, &its)) != KLECGC_OK) return s;
    WS(int, act, "act_all", S);
    TRY(cudaMemsetAsync(act, 0xff, S * sizeof(int), st));
    const Plan2D pl = plan_2d(fine_kind(ctx, false), ctx->nx, S);
    // A system whose FP64 Krylov vectors would stream from global memory
    // (pl.per_cta > 0) is solved on a thread-block cluster instead, by FP64
    // iterative refinement around FP32 PCG: the same FP64 residual test
    // ||b - M x||_2 <= rtol ||b||_2 in every step, so the same accuracy.
    Plan2D plc;
    if (ctx->prob.advection == 0 && (pl.per_cta > 0 || ctx->method2d == 3))
        plc = plan_2d(2, ctx->nx, S, true);
    WS(double, scr, "k2d_scratch", plc.cl.CL ? 0 : pl.scratch_doubles);
    ctx->launch(KLECGC_K_FINE, st, [&] {
        if (plc.cl.CL)
            launch_fine2d_mixed(plc, S, N, ctx->nx, J, dt * ctx->prob.reaction,
                                dt * ctx->prob.forcing, 0.0, 1, nullptr, ctx->u0, wdt,
                                ctx->kry_rtol_fine, kInnerRtol, ctx->kry_maxit, out, act, ifail,
                                its, nullptr, st);
        else
            launch_fine2d(pl, S, N, ctx->nx, J, dt * ctx->prob.reaction, dt * ctx->prob.forcing,
                          dt * ctx->prob.advection, 0.0,
                          1, nullptr, ctx->u0, wdt, ctx->kry_rtol_fine, ctx->kry_maxit, out, act,
                          ifail, its, scr, st);
    });
    TRY(cudaGetLastError());
    std::vector<int> hf;
    return krylov_read(ctx, S, ifail, its, st, &hf, capped);
}

bool nonlinear(const klecgc_ctx* ctx) {
    return ctx->prob.reaction_kind == 1 || ctx->prob.reaction_kind == 2;
}

// Nonlinear problem: coefficient field and the face weights a / h^2.
klecgc_status nl_weights(klecgc_ctx* ctx, const double* xi_d, int64_t S, cudaStream_t st,
                         double** a_out, double** wf_out) {
    double* a = nullptr;
    klecgc_status s = build_field(ctx, xi_d, S, st, &a);
    if (s != KLECGC_OK) return s;
    WS(double, wf, "wf_nl", S * (int64_t)ctx->nf);
    ctx->launch(KLECGC_K_FIELD, st, [&] { launch_face_weights(a, S, ctx->nf, 1.0 / (ctx->h * ctx->h), wf, st); });
    TRY(cudaGetLastError());
    *a_out = a;
    *wf_out = wf;
    return KLECGC_OK;
}

// Sequential Newton fine solution (N intervals of J steps of T/(N J)) into U
// (internal layout); *capped if a Newton step reached its iteration cap.
klecgc_status nl_sequential(klecgc_ctx* ctx, const double* wf, int64_t S, int N, int J,
                            double dt, double* U, cudaStream_t st, bool* capped) {
    WS(double, scr, "nl_seq_scratch", 4 * S * (int64_t)ctx->nx);
    WS(int, flag, "nl_seq_fail", S);
    TRY(cudaMemsetAsync(flag, 0, S * sizeof(int), st));
    ctx->launch(KLECGC_K_FINE, st, [&] {
        launch_sequential_newton(ctx->prob.reaction_kind, S, N, ctx->nx, J, dt, ctx->prob.reaction,
                                 ctx->prob.forcing, ctx->u0, wf, scr, U, flag, st);
    });
    TRY(cudaGetLastError());
    std::vector<int> h(S);
    TRY(cudaMemcpyAsync(h.data(), flag, S * sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    *capped = false;
    for (int v : h) *capped |= v != 0;
    return KLECGC_OK;
}

// alpha^{j/N} and alpha^{-j/N} / (N/2) tables in precision T.
template <typename T>
klecgc_status scale_tables(klecgc_ctx* ctx, int N, double alpha, cudaStream_t st, T** sc,
                           T** isc) {
    std::vector<T> a(N), b(N);
    for (int j = 0; j < N; ++j) {
        a[j] = (T)std::pow(alpha, (double)j / N);
        b[j] = (T)(std::pow(alpha, -(double)j / N) / (2 * N));  // 1/N and the transforms' 2 x 2
    }
    const char* n1 = sizeof(T) == 8 ? "scale64" : "scale32";
    const char* n2 = sizeof(T) == 8 ? "iscale64" : "iscale32";
    WS(T, d1, n1, N);
    WS(T, d2, n2, N);
    TRY(cudaMemcpyAsync(d1, a.data(), N * sizeof(T), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(d2, b.data(), N * sizeof(T), cudaMemcpyHostToDevice, st));
    *sc = d1;
    *isc = d2;
    return KLECGC_OK;
}

// Coarse sweep U^0_n = G(U^0_{n-1}), U^0_0 = u0 (the initial guess by G alone,
// Section 3.1): N backward-Euler steps of dT per sample into U (internal
// layout).  field: the coefficient a [S][nx+1] (1D) or the weights dT a / h^2
// [S][nf] (2D).
klecgc_status coarse_guess_internal(klecgc_ctx* ctx, int64_t S, int N, double dT,
                                    const double* field, double* U, cudaStream_t st) {
    const double react = ctx->prob.reaction, forcing = ctx->prob.forcing;
    if (ctx->dim == 1) {
        WS(FineCoef64, fc, "coarse64", S * (int64_t)(ctx->nx + 1));
        WS(double, scr, "seq_scratch", S * (int64_t)ctx->nx);
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_fine_factors(field, S, ctx->nx, ctx->h, dT, react, fc, nullptr, st); });
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_fine_sequential(S, N, ctx->nx, 1, dT * forcing, ctx->u0, fc, scr, U, st); });
    } else if (use_band(ctx, true)) {
        double* Bf = nullptr;
        klecgc_status s = band_factors_fine(ctx, field, S, dT, st, &Bf);
        if (s != KLECGC_OK) return s;
        WS(int, act, "act_all", S);
        WS(double, xs, "band_x", S * (int64_t)ctx->ns);
        TRY(cudaMemsetAsync(act, 0xff, S * sizeof(int), st));
        ctx->launch(KLECGC_K_GUESS, st, [&] {
            launch_band_fine(S, N, ctx->nx, 1, dT * react, dT * forcing, dT * ctx->prob.advection,
                             0.0, 1, nullptr, ctx->u0, field, Bf, xs, U, act, st);
        });
    } else {
        WS(int, act, "act_all", S);
        WS(int, gfail, "coarse_fail", S);
        TRY(cudaMemsetAsync(act, 0xff, S * sizeof(int), st));
        const Plan2D pl = plan_2d(fine_kind(ctx, false), ctx->nx, S);
        Plan2D plc;   // on a thread-block cluster where FP64 would stream (as the reference)
        if (ctx->prob.advection == 0 && (pl.per_cta > 0 || ctx->method2d == 3))
            plc = plan_2d(2, ctx->nx, S, true);
        WS(double, scr, "k2d_scratch_g", plc.cl.CL ? 0 : pl.scratch_doubles);
        // a guess needs no tight solve: its error only costs iterations
        ctx->launch(KLECGC_K_GUESS, st, [&] {
            if (plc.cl.CL)
                launch_fine2d_mixed(plc, S, N, ctx->nx, 1, dT * react, dT * forcing, 0.0, 1,
                                    nullptr, ctx->u0, field, ctx->kry_rtol_fine, kInnerRtol,
                                    ctx->kry_maxit, U, act, gfail, nullptr, nullptr, st);
            else
                launch_fine2d(pl, S, N, ctx->nx, 1, dT * react, dT * forcing,
                              dT * ctx->prob.advection, 0.0, 1, nullptr, ctx->u0,
                              field, ctx->kry_rtol_fine, ctx->kry_maxit, U, act, gfail, nullptr, scr, st);
        });
    }
    TRY(cudaGetLastError());
    return KLECGC_OK;
}

// Reads and clears the tensor-core guess's timeout flag (stream synchronized).
klecgc_status check_tc(klecgc_ctx* ctx, cudaStream_t st) {
    int h = 0;
    TRY(cudaMemcpyAsync(&h, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (h) {
        TRY(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), st));
        return fail(KLECGC_E_CUDA, "a tensor-core (tcgen05) pipeline timed out");
    }
    return KLECGC_OK;
}

// U^0 = ubar + psi(xi) W into U (internal layout [S][nx][N]).
klecgc_status gpc_guess_internal(klecgc_ctx* ctx, const double* xi_d, int64_t S, bool fp64,
                                 double* U, cudaStream_t st, bool pairs = false) {
    const int64_t NC = (int64_t)ctx->ns * ctx->N;
    if (fp64) {
        WS(double, psi, "psi64", S * ctx->P);
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_psi<double>(xi_d, S, ctx->M, ctx->degrees, ctx->P, psi, ctx->P, st); });
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_gemm<double>(S, NC, ctx->P, psi, ctx->P, 1, ctx->W, NC, 1, U, NC, false, ctx->ubar, st); });
    } else {
        // tcgen05 tensor cores, 3xTF32 split (FP32-level accuracy)
        WS(float, psi, "psi32", S * ctx->Kp);
        WS(float, psi_lo, "psi32lo", S * ctx->Kp);
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_psi<float>(xi_d, S, ctx->M, ctx->degrees, ctx->P, psi, ctx->Kp, st); });
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_split_tf32(psi, S * ctx->Kp, psi, psi_lo, st); });
        cudaError_t e = cudaSuccess;
        ctx->launch(KLECGC_K_GUESS, st, [&] {
            e = launch_guess_tc(S, NC, ctx->Kp, psi, psi_lo, ctx->W32t, ctx->W32t_lo, ctx->ubar,
                                pairs ? ctx->ubar_df : nullptr, U, ctx->tc_err, st);
        });
        TRY(e);
    }
    TRY(cudaGetLastError());
    return KLECGC_OK;
}

// ---------------------------------------------------------------- learned guess
klecgc_status mlp_alloc(klecgc_ctx* ctx) {
    MlpState& q = ctx->mlp;
    if (ctx->dim != 1 || nonlinear(ctx))
        return fail(KLECGC_E_UNSUPPORTED, "the learned guess is for the linear 1D problem only");
    if (q.theta) return KLECGC_OK;
    const int W = 256;
    q.sizes[0] = ctx->M;
    q.sizes[1] = q.sizes[2] = q.sizes[3] = W;
    q.sizes[4] = 64 * ctx->N;
    q.D = q.sizes[4];
    int64_t k = 0;
    for (int l = 0; l < 4; ++l) {
        q.woff[l] = k;
        k += (int64_t)q.sizes[l + 1] * q.sizes[l];
        q.boff[l] = k;
        k += q.sizes[l + 1];
    }
    q.P = k;
    TRY(ctx->alloc_owned(&q.theta, q.P));
    TRY(ctx->alloc_owned(&q.thb, q.P));
    TRY(ctx->alloc_owned(&q.m, q.P));
    TRY(ctx->alloc_owned(&q.v, q.P));
    TRY(ctx->alloc_owned(&q.grad, q.P));
    TRY(ctx->alloc_owned(&q.mean, q.D));
    TRY(ctx->alloc_owned(&q.stdv, q.D));
    TRY(ctx->alloc_owned(&q.inv_std, q.D));
    std::vector<float> zero(q.D, 0.f), one(q.D, 1.f);
    TRY(cudaMemcpy(q.mean, zero.data(), q.D * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(q.stdv, one.data(), q.D * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(q.inv_std, one.data(), q.D * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemset(q.theta, 0, q.P * 4));
    TRY(cudaMemset(q.thb, 0, q.P * 2));
    return KLECGC_OK;
}

struct MlpBuffers {
    float* Z[3];
    __nv_bfloat16* A[3];
    float* dZ[2];
    __nv_bfloat16* dZb[2];
};

klecgc_status mlp_buffers(klecgc_ctx* ctx, int B, MlpBuffers* b) {
    const int W = ctx->mlp.sizes[1];
    const char* zn[3] = {"mlp_Z0", "mlp_Z1", "mlp_Z2"};
    const char* an[3] = {"mlp_A0", "mlp_A1", "mlp_A2"};
    for (int l = 0; l < 3; ++l) {
        WS(float, z, zn[l], (size_t)B * W);
        WS(__nv_bfloat16, a, an[l], (size_t)B * W);
        b->Z[l] = z;
        b->A[l] = a;
    }
    WS(float, d0, "mlp_dZ0", (size_t)B * W);
    WS(float, d1, "mlp_dZ1", (size_t)B * W);
    WS(__nv_bfloat16, e0, "mlp_dZb0", (size_t)B * W);
    WS(__nv_bfloat16, e1, "mlp_dZb1", (size_t)B * W);
    b->dZ[0] = d0;
    b->dZ[1] = d1;
    b->dZb[0] = e0;
    b->dZb[1] = e1;
    return KLECGC_OK;
}

// One GEMM of the network: C = op(A) op(B) (op = transpose when ta / tb;
// A(m,k) = ta ? A[k lda + m] : A[m lda + k], B(k,n) = tb ? B[n ldb + k] : B[k ldb + n]).
// On the tcgen05 tensor cores when the shape allows TMA (K-major operands,
// transposed into scratch where op needs it), else on the warp-level MMA
// kernel (the first layer, with K = M = 10, and short tails).
klecgc_status mlp_gemm(klecgc_ctx* ctx, bool ta, bool tb, int M, int N, int K,
                       const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                       const float* bias, const float* zmask, int ldz, float* C, int ldc,
                       __nv_bfloat16* Cb, int ldcb, bool relu, cudaStream_t st) {
    const __nv_bfloat16* Ak = A;
    const __nv_bfloat16* Bk = B;
    int la = lda, lb = ldb;
    bool tc = ctx->mlp_tc && M >= 64 && N >= 32 && K >= 64 && (K % 8) == 0;
    if (tc && ta) {
        WS(__nv_bfloat16, t, "mlp_tA", (size_t)M * K);
        launch_transpose_bf16(A, K, M, lda, t, st);   // [K][M] -> [M][K]
        Ak = t;
        la = K;
    }
    if (tc && !tb) {
        WS(__nv_bfloat16, t, "mlp_tB", (size_t)N * K);
        launch_transpose_bf16(B, K, N, ldb, t, st);   // [K][N] -> [N][K]
        Bk = t;
        lb = K;
    }
    if (tc && gemm_bf16_tc_ok(M, N, K, Ak, la, Bk, lb)) {
        TRY(launch_gemm_bf16_tc(M, N, K, Ak, la, Bk, lb, bias, zmask, ldz, C, ldc, Cb, ldcb, relu,
                                ctx->tc_err, st));
        return KLECGC_OK;
    }
    launch_gemm_bf16(ta, tb, M, N, K, A, lda, B, ldb, bias, zmask, ldz, C, ldc, Cb, ldcb, relu, st);
    return KLECGC_OK;
}

// Y = net(X), X BF16 [B][M]; hidden pre-activations and activations kept in b.
klecgc_status mlp_forward(klecgc_ctx* ctx, int B, const __nv_bfloat16* X, const MlpBuffers& b,
                          float* Y, cudaStream_t st) {
    klecgc_status s = KLECGC_OK;
    MlpState& q = ctx->mlp;
    const __nv_bfloat16* in = X;
    int kin = q.sizes[0];
    for (int l = 0; l < 4; ++l) {
        const int out = q.sizes[l + 1];
        const __nv_bfloat16* W = q.thb + q.woff[l];
        const float* bias = q.theta + q.boff[l];
        if (l < 3) {
            ctx->launch(KLECGC_K_GUESS, st, [&] {
                s = mlp_gemm(ctx, false, true, B, out, kin, in, kin, W, kin, bias, nullptr, 0,
                             b.Z[l], out, b.A[l], out, true, st);
            });
            in = b.A[l];
            kin = out;
        } else {
            ctx->launch(KLECGC_K_GUESS, st, [&] {
                s = mlp_gemm(ctx, false, true, B, out, kin, in, kin, W, kin, bias, nullptr, 0, Y,
                             out, nullptr, 0, false, st);
            });
        }
        if (s != KLECGC_OK) return s;
    }
    return KLECGC_OK;
}

// Gradient of the loss w.r.t. all parameters into q.grad, from dY (FP32 and BF16).
klecgc_status mlp_backward(klecgc_ctx* ctx, int B, const __nv_bfloat16* X, const MlpBuffers& b,
                           const float* dY, const __nv_bfloat16* dYb, cudaStream_t st) {
    klecgc_status s = KLECGC_OK;
    MlpState& q = ctx->mlp;
    const float* dZf = dY;
    const __nv_bfloat16* dZb = dYb;
    for (int l = 3; l >= 0; --l) {
        const int out = q.sizes[l + 1], kin = q.sizes[l];
        const __nv_bfloat16* Ain = l == 0 ? X : b.A[l - 1];
        ctx->launch(KLECGC_K_GUESS, st, [&] {
            s = mlp_gemm(ctx, true, false, out, kin, B, dZb, out, Ain, kin, nullptr, nullptr, 0,
                         q.grad + q.woff[l], kin, nullptr, 0, false, st);
        });
        if (s != KLECGC_OK) return s;
        ctx->launch(KLECGC_K_GUESS, st, [&] { launch_colsum(B, out, dZf, q.grad + q.boff[l], st); });
        if (l > 0) {
            const int nb = l & 1;
            ctx->launch(KLECGC_K_GUESS, st, [&] {
                s = mlp_gemm(ctx, false, false, B, kin, out, dZb, out, q.thb + q.woff[l], kin,
                             nullptr, b.Z[l - 1], kin, b.dZ[nb], kin, b.dZb[nb], kin, false, st);
            });
            if (s != KLECGC_OK) return s;
            dZf = b.dZ[nb];
            dZb = b.dZb[nb];
        }
    }
    return KLECGC_OK;
}

// Learned guess of S samples into U (internal layout [S][nx][N]); *finite
// reports whether every network output was finite.
klecgc_status mlp_guess_internal(klecgc_ctx* ctx, const double* xi_d, int64_t S, double* U,
                                 cudaStream_t st, bool* finite) {
    MlpState& q = ctx->mlp;
    const int B = (int)S;
    MlpBuffers b;
    klecgc_status s = mlp_buffers(ctx, B, &b);
    if (s != KLECGC_OK) return s;
    WS(__nv_bfloat16, X, "mlp_X", (size_t)B * q.sizes[0]);
    WS(float, Y, "mlp_Y", (size_t)B * q.D);
    ctx->launch(KLECGC_K_GUESS, st, [&] {
        launch_mlp_gather(B, q.sizes[0], q.D, nullptr, 0, xi_d, nullptr, nullptr, nullptr, X,
                          nullptr, st);
    });
    {
        const klecgc_status ms_ = mlp_forward(ctx, B, X, b, Y, st);
        if (ms_ != KLECGC_OK) return ms_;
    }
    if (q.residual) {
        // U0 = gPC surrogate guess (tensor-core contraction, FP32-accurate) +
        // the network's correction
        if ((s = gpc_guess_internal(ctx, xi_d, S, false, U, st)) != KLECGC_OK) return s;
    }
    ctx->launch(KLECGC_K_GUESS, st, [&] { launch_upsample(S, ctx->N, ctx->nx, Y, q.mean, q.stdv, U, q.residual, st); });
    WS(int, flag, "mlp_flag", 1);
    TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
    launch_nonfinite_f32((int64_t)B * q.D, Y, flag, st);
    int h = 0;
    TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    *finite = h == 0;
    return KLECGC_OK;
}

template <typename T>
klecgc_status stage_any(klecgc_ctx* ctx, const T* user, size_t count, const char* name,
                        cudaStream_t st, const T** out) {
    return stage_in(ctx, user, count, name, st, out);
}

klecgc_status check_xi_finite(klecgc_ctx* ctx, const double* xi_d, int64_t n, cudaStream_t st,
                              bool* finite) {
    WS(int, flag, "flag", 1);
    TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
    ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_nonfinite_flag(xi_d, n, flag, st); });
    int h = 0;
    TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    *finite = (h == 0);
    return KLECGC_OK;
}

// Copies an internal [S][nx][N] batch to the caller's [S][N][nx] array.
klecgc_status export_batch(klecgc_ctx* ctx, const double* U_int, int64_t S, int N, double* out,
                           cudaStream_t st) {
    const int nx = ctx->ns;
    if (is_device_ptr(out)) {
        ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_transpose(U_int, out, S, nx, N, st); });
        TRY(cudaGetLastError());
    } else {
        WS(double, tmp, "export", S * (int64_t)nx * N);
        ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_transpose(U_int, tmp, S, nx, N, st); });
        TRY(cudaGetLastError());
        TRY(cudaMemcpyAsync(out, tmp, S * (size_t)nx * N * sizeof(double), cudaMemcpyDeviceToHost,
                            st));
    }
    return KLECGC_OK;
}

// Reads a caller [S][N][nx] array into internal layout.
klecgc_status import_batch(klecgc_ctx* ctx, const double* user, int64_t S, int N, double* U_int,
                           cudaStream_t st) {
    const double* src = nullptr;
    klecgc_status s = stage_in(ctx, user, (size_t)S * ctx->ns * N, "import", st, &src);
    if (s != KLECGC_OK) return s;
    ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_transpose(src, U_int, S, N, ctx->ns, st); });
    TRY(cudaGetLastError());
    return KLECGC_OK;
}

}  // namespace

extern "C" {

const char* klecgc_status_string(klecgc_status s) {
    switch (s) {
        case KLECGC_OK: return "ok";
        case KLECGC_E_INVALID_ARG: return "invalid argument";
        case KLECGC_E_OUT_OF_MEMORY: return "out of device memory";
        case KLECGC_E_NOT_CONVERGED: return "not converged within kmax iterations";
        case KLECGC_E_NONFINITE: return "non-finite value";
        case KLECGC_E_CUDA: return "CUDA runtime error";
        case KLECGC_E_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char* klecgc_last_error(void) { return g_last_error.c_str(); }

void klecgc_free(klecgc_ctx* ctx) {
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->device);
    delete ctx;
    cudaSetDevice(cur);
}

// ------------------------------------------------------------ save / load
// File: magic, version, klecgc_problem, sizes, then the device tables as
// raw arrays in native byte order (basis, u0, degrees, ubar, W) and, when a network
// is set, its parameters and output normalization.
}  // extern "C"
namespace {
constexpr char kMagic[8] = {'K', 'L', 'E', 'C', 'G', 'C', 'v', '1'};
constexpr int32_t kVersion = 6;   // 5: learned-guess mode; 6: autotuner choices

struct FileHead {
    char magic[8];
    int32_t version;
    int32_t dim, nx, N, J, M, P, MQ, p, ns, nf;
    int32_t mlp_ready, kry_maxit;
    double h, dT, lambda_sum, lambda_kept, kry_rtol_fine, kry_rtol_cgc;
    int64_t mlp_P;
    int32_t mlp_D, method2d;
    int32_t mlp_residual, pad;
};

template <typename T>
bool put_dev(FILE* f, const T* d, size_t n) {
    std::vector<T> h(n);
    if (n && cudaMemcpy(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return std::fwrite(h.data(), sizeof(T), n, f) == n;
}

template <typename T>
klecgc_status get_dev(FILE* f, klecgc_ctx* ctx, T** d, size_t n) {
    std::vector<T> h(n);
    if (std::fread(h.data(), sizeof(T), n, f) != n) return fail(KLECGC_E_INVALID_ARG, "truncated file");
    TRY(ctx->alloc_owned(d, n));
    TRY(cudaMemcpy(*d, h.data(), n * sizeof(T), cudaMemcpyHostToDevice));
    return KLECGC_OK;
}
}  // namespace
extern "C" {

klecgc_status klecgc_save(const klecgc_ctx* ctx, const char* path) {
    set_error("");
    if (!ctx || !path || !ctx->W) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(KLECGC_E_INVALID_ARG, std::string("cannot open ") + path);
    FileHead hd{};
    std::memcpy(hd.magic, kMagic, 8);
    hd.version = kVersion;
    hd.dim = ctx->dim;
    hd.nx = ctx->nx;
    hd.N = ctx->N;
    hd.J = ctx->J;
    hd.M = ctx->M;
    hd.P = ctx->P;
    hd.MQ = ctx->MQ;
    hd.p = ctx->p;
    hd.ns = ctx->ns;
    hd.nf = ctx->nf;
    hd.mlp_ready = ctx->mlp.ready ? 1 : 0;
    hd.kry_maxit = ctx->kry_maxit;
    hd.method2d = ctx->method2d;
    hd.h = ctx->h;
    hd.dT = ctx->dT;
    hd.lambda_sum = ctx->lambda_sum;
    hd.lambda_kept = ctx->lambda_kept;
    hd.kry_rtol_fine = ctx->kry_rtol_fine;
    hd.kry_rtol_cgc = ctx->kry_rtol_cgc;
    hd.mlp_P = ctx->mlp.ready ? ctx->mlp.P : 0;
    hd.mlp_D = ctx->mlp.ready ? ctx->mlp.D : 0;
    hd.mlp_residual = ctx->mlp.residual ? 1 : 0;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->device);
    const size_t NC = (size_t)ctx->ns * ctx->N;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
              std::fwrite(&ctx->prob, sizeof(ctx->prob), 1, f) == 1 &&
              put_dev(f, ctx->basis, (size_t)ctx->M * ctx->nf) && put_dev(f, ctx->u0, ctx->ns) &&
              put_dev(f, ctx->degrees, (size_t)ctx->P * ctx->M) && put_dev(f, ctx->ubar, NC) &&
              put_dev(f, ctx->W, (size_t)ctx->P * NC);
    if (ok && ctx->mlp.ready)
        ok = put_dev(f, ctx->mlp.theta, ctx->mlp.P) && put_dev(f, ctx->mlp.mean, ctx->mlp.D) &&
             put_dev(f, ctx->mlp.stdv, ctx->mlp.D);
    if (ok) {
        // the autotuner's choices, so that a loaded context reruns the same
        // kernels (and reproduces solves bit for bit)
        const std::string tj = tune_json(ctx);
        const int64_t len = (int64_t)tj.size();
        ok = std::fwrite(&len, sizeof(len), 1, f) == 1 &&
             (len == 0 || std::fwrite(tj.data(), 1, (size_t)len, f) == (size_t)len);
    }
    cudaSetDevice(cur);
    ok = (std::fclose(f) == 0) && ok;
    return ok ? KLECGC_OK : fail(KLECGC_E_CUDA, std::string("writing ") + path + " failed");
}

klecgc_status klecgc_load(const char* path, klecgc_ctx** out, void* stream) {
    set_error("");
    if (!path || !out) return fail(KLECGC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(KLECGC_E_INVALID_ARG, std::string("cannot open ") + path);
    struct Closer {
        FILE* f;
        ~Closer() { std::fclose(f); }
    } closer{f};
    FileHead hd{};
    klecgc_problem pr{};
    if (std::fread(&hd, sizeof(hd), 1, f) != 1 || std::memcmp(hd.magic, kMagic, 8) != 0 ||
        hd.version != kVersion || std::fread(&pr, sizeof(pr), 1, f) != 1)
        return fail(KLECGC_E_INVALID_ARG, std::string(path) + " is not a klecgc context file");
    const bool sane = (hd.dim == 1 || hd.dim == 2) && hd.nx >= 1 && hd.nx <= 1 << 20 &&
                      pow2_in_range(hd.N) && hd.M >= 1 && hd.M <= 4096 && hd.P >= 1 &&
                      hd.MQ >= 1 && hd.ns == (hd.dim == 1 ? hd.nx : hd.nx * hd.nx) &&
                      hd.nf == (hd.dim == 1 ? hd.nx + 1 : 2 * hd.nx * (hd.nx + 1)) &&
                      pr.dim == hd.dim && pr.nx == hd.nx && pr.N == hd.N && pr.M == hd.M &&
                      (int64_t)hd.P * hd.ns * hd.N < ((int64_t)1 << 36) &&
                      (hd.mlp_ready == 0 || (hd.mlp_P > 0 && hd.mlp_D == 64 * hd.N && hd.dim == 1));
    if (!sane) return fail(KLECGC_E_INVALID_ARG, std::string(path) + ": inconsistent header");
    cudaStream_t st = (cudaStream_t)stream;
    klecgc_ctx* ctx = new klecgc_ctx();
    auto bail = [&](klecgc_status s) {
        delete ctx;
        return s;
    };
    ctx->prob = pr;
    cudaGetDevice(&ctx->device);
    ctx->dim = hd.dim;
    ctx->nx = hd.nx;
    ctx->N = hd.N;
    ctx->J = hd.J;
    ctx->M = hd.M;
    ctx->P = hd.P;
    ctx->MQ = hd.MQ;
    ctx->p = hd.p;
    ctx->ns = hd.ns;
    ctx->nf = hd.nf;
    ctx->h = hd.h;
    ctx->dT = hd.dT;
    ctx->lambda_sum = hd.lambda_sum;
    ctx->lambda_kept = hd.lambda_kept;
    ctx->kry_rtol_fine = hd.kry_rtol_fine;
    ctx->kry_rtol_cgc = hd.kry_rtol_cgc;
    ctx->kry_maxit = hd.kry_maxit;
    ctx->method2d = hd.method2d >= 0 && hd.method2d <= 3 ? hd.method2d : 0;
    ctx->mlp.residual = hd.mlp_residual == 1;
    const size_t NC = (size_t)ctx->ns * ctx->N;
    klecgc_status s;
    if ((s = get_dev(f, ctx, &ctx->basis, (size_t)ctx->M * ctx->nf)) != KLECGC_OK ||
        (s = get_dev(f, ctx, &ctx->u0, ctx->ns)) != KLECGC_OK ||
        (s = get_dev(f, ctx, &ctx->degrees, (size_t)ctx->P * ctx->M)) != KLECGC_OK ||
        (s = get_dev(f, ctx, &ctx->ubar, NC)) != KLECGC_OK ||
        (s = get_dev(f, ctx, &ctx->W, (size_t)ctx->P * NC)) != KLECGC_OK)
        return bail(s);
    ctx->Kp = guess_tc_k_padded(ctx->P);
    if (ctx->alloc_owned(&ctx->W32, (size_t)ctx->P * NC) != cudaSuccess ||
        ctx->alloc_owned(&ctx->W32t, (size_t)ctx->Kp * NC) != cudaSuccess ||
        ctx->alloc_owned(&ctx->W32t_lo, (size_t)ctx->Kp * NC) != cudaSuccess ||
        ctx->alloc_owned(&ctx->tc_err, 1) != cudaSuccess)
        return bail(fail(KLECGC_E_OUT_OF_MEMORY, "W32"));
    if (cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), st) != cudaSuccess)
        return bail(fail(KLECGC_E_CUDA, "memset"));
    launch_to_float(ctx->W, ctx->W32, (int64_t)ctx->P * NC, st);
    launch_pad_transpose(ctx->W32, ctx->P, NC, ctx->Kp, ctx->W32t, st);
    launch_split_tf32(ctx->W32t, (int64_t)ctx->Kp * NC, ctx->W32t, ctx->W32t_lo, st);
    if (ctx->alloc_owned(&ctx->ubar_df, NC) != cudaSuccess)
        return bail(fail(KLECGC_E_OUT_OF_MEMORY, "ubar pairs"));
    cudaMemcpyAsync(ctx->ubar_df, ctx->ubar, NC * sizeof(double), cudaMemcpyDeviceToDevice, st);
    launch_to_pairs(reinterpret_cast<double*>(ctx->ubar_df), (int64_t)NC, st);
    if (hd.mlp_ready) {
        if ((s = mlp_alloc(ctx)) != KLECGC_OK) return bail(s);
        MlpState& q = ctx->mlp;
        if (q.P != hd.mlp_P || q.D != hd.mlp_D)
            return bail(fail(KLECGC_E_INVALID_ARG, "network size does not match the problem"));
        std::vector<float> th(q.P), mu(q.D), sd(q.D), inv(q.D);
        if (std::fread(th.data(), 4, q.P, f) != (size_t)q.P || std::fread(mu.data(), 4, q.D, f) != (size_t)q.D ||
            std::fread(sd.data(), 4, q.D, f) != (size_t)q.D)
            return bail(fail(KLECGC_E_INVALID_ARG, "truncated file"));
        for (int c = 0; c < q.D; ++c) {
            if (!(sd[c] > 0)) return bail(fail(KLECGC_E_INVALID_ARG, "bad output normalization"));
            inv[c] = 1.f / sd[c];
        }
        if (cudaMemcpy(q.theta, th.data(), q.P * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(q.mean, mu.data(), q.D * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(q.stdv, sd.data(), q.D * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(q.inv_std, inv.data(), q.D * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(KLECGC_E_CUDA, "network upload"));
        launch_f32_to_bf16(q.P, q.theta, q.thb, st);
        q.ready = true;
    }
    {
        int64_t len = -1;
        if (std::fread(&len, sizeof(len), 1, f) != 1 || len < 0 || len > (1 << 24))
            return bail(fail(KLECGC_E_INVALID_ARG, "truncated file (autotuner choices)"));
        std::string tj((size_t)len, '\0');
        if (len && std::fread(&tj[0], 1, (size_t)len, f) != (size_t)len)
            return bail(fail(KLECGC_E_INVALID_ARG, "truncated file (autotuner choices)"));
        tune_parse(ctx, tj);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return bail(fail(KLECGC_E_CUDA, "upload"));
    *out = ctx;
    return KLECGC_OK;
}

klecgc_status klecgc_kl_basis(int32_t dim, double corr_len, double sigma, int32_t M,
                              const double* x, int64_t npts, double* out, double* lambda_out) {
    set_error("");
    if (dim != 1 && dim != 2) return fail(KLECGC_E_UNSUPPORTED, "dim must be 1 or 2");
    if (M < 1 || M > (dim == 1 ? 65536 : 1024) || npts < 0 || (npts > 0 && (!x || !out)) ||
        !(corr_len > 0) || !std::isfinite(corr_len) || !(sigma >= 0) || !std::isfinite(sigma))
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    // the expressions of klecgc_setup's basis, so the values are identical
    if (dim == 1) {
        std::vector<double> lam, om;
        std::vector<int> par;
        kl_modes_1d(corr_len, sigma, M, lam, om, par);
        for (int m = 0; m < M; ++m) {
            for (int64_t i = 0; i < npts; ++i)
                out[(size_t)m * npts + i] = std::sqrt(lam[m]) * kl_phi_1d(x[i], om[m], par[m]);
            if (lambda_out) lambda_out[m] = lam[m];
        }
    } else {
        std::vector<double> lam, mu, om;
        std::vector<int> mi, mj, par;
        kl_modes_2d(corr_len, sigma, M, lam, mi, mj, mu, om, par);
        for (int m = 0; m < M; ++m) {
            const double sl = std::sqrt(lam[m]);
            for (int64_t i = 0; i < npts; ++i)
                out[(size_t)m * npts + i] = sl * kl_phi_1d(x[2 * i], om[mi[m]], par[mi[m]]) *
                                            kl_phi_1d(x[2 * i + 1], om[mj[m]], par[mj[m]]);
            if (lambda_out) lambda_out[m] = lam[m];
        }
    }
    return KLECGC_OK;
}

klecgc_status klecgc_gpc_indices(int32_t M, int32_t p, int32_t* out, int64_t capacity,
                                 int64_t* P_out) {
    set_error("");
    if (M < 1 || p < 0 || !P_out || capacity < 0) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    // P = C(M + p, p), built up as C(M + d, d) = C(M + d - 1, d - 1) (M + d) / d
    int64_t P = 1;
    for (int d = 1; d <= p; ++d) {
        P = P * (M + d) / d;
        if (P > (int64_t)1 << 24) return fail(KLECGC_E_UNSUPPORTED, "more than 2^24 basis functions");
    }
    if ((int64_t)M * P > (int64_t)1 << 28)
        return fail(KLECGC_E_UNSUPPORTED, "more than 2^28 multi-index entries");
    *P_out = P;
    if (!out) return KLECGC_OK;
    if (capacity < P) return fail(KLECGC_E_INVALID_ARG, "capacity below P");
    const std::vector<int> deg = gpc_multi_indices(M, p);
    std::copy(deg.begin(), deg.end(), out);
    return KLECGC_OK;
}

klecgc_status klecgc_info(const klecgc_ctx* ctx, klecgc_info_t* out) {
    if (!ctx || !out) return fail(KLECGC_E_INVALID_ARG, "NULL argument");
    out->nx = ctx->nx;
    out->N = ctx->N;
    out->J = ctx->J;
    out->M = ctx->M;
    out->P = ctx->P;
    out->MQ = ctx->MQ;
    out->lambda_sum = ctx->lambda_sum;
    out->lambda_kept = ctx->lambda_kept;
    out->n_unknowns = ctx->ns;
    out->device = ctx->device;
    return KLECGC_OK;
}

klecgc_status klecgc_set_krylov(klecgc_ctx* ctx, double rtol_fine, double rtol_cgc,
                                int32_t maxit) {
    set_error("");
    if (!ctx || !(rtol_fine > 0 && rtol_fine < 1) || !(rtol_cgc > 0 && rtol_cgc < 1) || maxit < 1)
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    ctx->kry_rtol_fine = rtol_fine;
    ctx->kry_rtol_cgc = rtol_cgc;
    ctx->kry_maxit = maxit;
    return KLECGC_OK;
}

klecgc_status klecgc_set_scratch_limit(klecgc_ctx* ctx, int64_t bytes) {
    set_error("");
    if (!ctx || bytes < 0) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    ctx->ws_limit = (size_t)bytes;
    return KLECGC_OK;
}

klecgc_status klecgc_set_2d_method(klecgc_ctx* ctx, int32_t method) {
    set_error("");
    if (!ctx || method < 0 || method > 3) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (method == 2 && (ctx->dim != 2 || ctx->nx > kBandMaxNx))
        return fail(KLECGC_E_UNSUPPORTED, "banded LU: 2D grids with nx <= 64");
    if (method == 3 && ctx->dim != 2) return fail(KLECGC_E_UNSUPPORTED, "clusters: 2D only");
    ctx->method2d = method;
    return KLECGC_OK;
}

klecgc_status klecgc_set_tuning(klecgc_ctx* ctx, int32_t mode, const char* cache_path) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    if (mode != 0 && mode != 1) return fail(KLECGC_E_INVALID_ARG, "tuning mode must be 0 or 1");
    ctx->tune_mode = mode;
    ctx->tune_path = cache_path ? cache_path : "";
    tune_load(ctx);
    return KLECGC_OK;
}

klecgc_status klecgc_tuning_report(const klecgc_ctx* ctx, char* buf, int64_t capacity,
                                   int64_t* length) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    const std::string j = tune_json(ctx);
    if (length) *length = (int64_t)j.size();
    if (buf && capacity > 0) {
        const size_t n = std::min<size_t>(j.size(), (size_t)capacity - 1);
        std::memcpy(buf, j.data(), n);
        buf[n] = 0;
    }
    return KLECGC_OK;
}

klecgc_status klecgc_set_loop(klecgc_ctx* ctx, int32_t mode) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    if (mode != 0 && mode != 1) return fail(KLECGC_E_INVALID_ARG, "loop mode must be 0 or 1");
    ctx->loop_mode = mode;
    return KLECGC_OK;
}

klecgc_status klecgc_krylov_stats(const klecgc_ctx* ctx, int64_t* its_fine, int64_t* its_cgc) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    if (its_fine) *its_fine = (int64_t)ctx->kry_it_fine;
    if (its_cgc) *its_cgc = (int64_t)ctx->kry_it_cgc;
    return KLECGC_OK;
}

klecgc_status klecgc_profile_enable(klecgc_ctx* ctx, int32_t timing) {
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    ctx->prof_collect();
    ctx->prof_timing = timing != 0;
    for (int i = 0; i < KLECGC_K_COUNT; ++i) {
        ctx->prof_launches[i] = 0;
        ctx->prof_ms[i] = 0.0;
    }
    return KLECGC_OK;
}

klecgc_status klecgc_profile_read(const klecgc_ctx* ctx, klecgc_profile_t* out) {
    if (!ctx || !out) return fail(KLECGC_E_INVALID_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    out->n_classes = KLECGC_K_COUNT;
    for (int i = 0; i < KLECGC_K_COUNT; ++i) {
        out->launches[i] = ctx->prof_launches[i];
        out->ms[i] = ctx->prof_ms[i];
    }
    return KLECGC_OK;
}

klecgc_status klecgc_setup(const klecgc_problem* pr, const double* xi_train, klecgc_ctx** out,
                           void* stream) {
    set_error("");
    if (!pr || !out || !xi_train) return fail(KLECGC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (pr->dim != 1 && pr->dim != 2) return fail(KLECGC_E_UNSUPPORTED, "dim must be 1 or 2");
    if (pr->dim == 2 && pr->nx > 2047) return fail(KLECGC_E_UNSUPPORTED, "2D needs nx <= 2047");
    if (pr->nx < 1 || pr->M < 1 || pr->gpc_degree < 0 || pr->n_train < 2 || !(pr->T > 0) ||
        !(pr->sigma >= 0) || !(pr->corr_len > 0) || !(pr->eps_kl >= 0) || pr->J < 1 ||
        !(pr->reaction >= 0) || !std::isfinite(pr->forcing) || pr->u0_kind < 0 ||
        pr->u0_kind > 2 || pr->reaction_kind < 0 || pr->reaction_kind > 2 || pr->cgc_newton < 0 ||
        !(pr->advection >= 0) || !std::isfinite(pr->advection))
        return fail(KLECGC_E_INVALID_ARG, "problem field out of range");
    if ((pr->u0_kind == 2 || pr->advection > 0) && pr->dim != 2)
        return fail(KLECGC_E_UNSUPPORTED, "u0_kind 2 and advection are 2D only");
    if (pr->advection > 0 && pr->reaction_kind != 0)
        return fail(KLECGC_E_UNSUPPORTED, "advection with a linear reaction only");
    if (pr->reaction_kind != 0 && pr->dim != 1)
        return fail(KLECGC_E_UNSUPPORTED, "the nonlinear problems are 1D only");
    if (!pow2_in_range(pr->N)) return fail(KLECGC_E_UNSUPPORTED, "N must be a power of 2 in [2, 64]");
    cudaStream_t st = (cudaStream_t)stream;
    klecgc_ctx* ctx = new klecgc_ctx();
    ctx->prob = *pr;
    cudaGetDevice(&ctx->device);
    ctx->nx = pr->nx;
    ctx->dim = pr->dim;
    ctx->ns = pr->dim == 1 ? pr->nx : pr->nx * pr->nx;
    ctx->nf = pr->dim == 1 ? pr->nx + 1 : 2 * pr->nx * (pr->nx + 1);
    ctx->N = pr->N;
    ctx->J = pr->J;
    ctx->M = pr->M;
    ctx->p = pr->gpc_degree;
    ctx->h = 1.0 / (pr->nx + 1);
    ctx->dT = pr->T / pr->N;
    auto bail = [&](klecgc_status s) {
        delete ctx;
        return s;
    };
#define STRY(expr)                                                                          \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? KLECGC_E_OUT_OF_MEMORY       \
                                                             : KLECGC_E_CUDA,               \
                             std::string(#expr) + ": " + cudaGetErrorString(e_)));          \
    } while (0)
#define SCHK(expr)                          \
    do {                                    \
        klecgc_status s_ = (expr);          \
        if (s_ != KLECGC_OK) return bail(s_); \
    } while (0)
    const int nx = ctx->nx, nf = ctx->nf, ns = ctx->ns, N = ctx->N, M = ctx->M, nt = pr->n_train;
    const int64_t NC = (int64_t)ns * N;
    const double pi = 3.14159265358979323846, h = ctx->h;

    // 1. input KL basis at the faces, initial value, gPC multi-indices
    std::vector<double> basis((size_t)M * nf), u0(ns);
    if (ctx->dim == 1) {
        std::vector<double> lam, om;
        std::vector<int> par;
        kl_modes_1d(pr->corr_len, pr->sigma, M, lam, om, par);
        for (int m = 0; m < M; ++m)
            for (int f = 0; f < nf; ++f)
                basis[(size_t)m * nf + f] = std::sqrt(lam[m]) * kl_phi_1d((f + 0.5) * h, om[m], par[m]);
        for (int i = 0; i < nx; ++i) u0[i] = pr->u0_kind == 0 ? std::sin(pi * (i + 1) * h) : 0.0;
    } else {
        // separable modes sigma^2 mu_i mu_j, phi_i(x1) phi_j(x2); x-faces
        // [nx][nx+1] at ((fx+1/2)h, (iy+1)h), then y-faces [nx+1][nx] at
        // ((ix+1)h, (fy+1/2)h)
        std::vector<double> lam;
        std::vector<int> mi, mj;
        std::vector<double> mu, om;
        std::vector<int> par;
        kl_modes_2d(pr->corr_len, pr->sigma, M, lam, mi, mj, mu, om, par);
        const int nxf = nx * (nx + 1);
        for (int m = 0; m < M; ++m) {
            const double sl = std::sqrt(lam[m]);
            double* bm = basis.data() + (size_t)m * nf;
            for (int iy = 0; iy < nx; ++iy)
                for (int fx = 0; fx <= nx; ++fx)
                    bm[iy * (nx + 1) + fx] = sl * kl_phi_1d((fx + 0.5) * h, om[mi[m]], par[mi[m]]) *
                                             kl_phi_1d((iy + 1) * h, om[mj[m]], par[mj[m]]);
            for (int fy = 0; fy <= nx; ++fy)
                for (int ix = 0; ix < nx; ++ix)
                    bm[nxf + fy * nx + ix] = sl * kl_phi_1d((ix + 1) * h, om[mi[m]], par[mi[m]]) *
                                             kl_phi_1d((fy + 0.5) * h, om[mj[m]], par[mj[m]]);
        }
        for (int iy = 0; iy < nx; ++iy)
            for (int ix = 0; ix < nx; ++ix)
                u0[iy * nx + ix] =
                    pr->u0_kind == 0   ? std::sin(pi * (ix + 1) * h) * std::sin(pi * (iy + 1) * h)
                    : pr->u0_kind == 2 ? std::sin(pi * (ix + 1) * h) * std::sin(2 * pi * (iy + 1) * h)
                                       : 0.0;
    }
    std::vector<int> deg = gpc_multi_indices(M, ctx->p);
    ctx->P = (int)(deg.size() / M);
    const int P = ctx->P;
    STRY(ctx->alloc_owned(&ctx->basis, basis.size()));
    STRY(ctx->alloc_owned(&ctx->u0, ns));
    STRY(ctx->alloc_owned(&ctx->degrees, deg.size()));
    STRY(cudaMemcpyAsync(ctx->basis, basis.data(), basis.size() * 8, cudaMemcpyHostToDevice, st));
    STRY(cudaMemcpyAsync(ctx->u0, u0.data(), ns * 8, cudaMemcpyHostToDevice, st));
    STRY(cudaMemcpyAsync(ctx->degrees, deg.data(), deg.size() * 4, cudaMemcpyHostToDevice, st));

    // 2. snapshots: sequential fine solution of every training sample
    const double* xi_d = nullptr;
    SCHK(stage_in(ctx, xi_train, (size_t)nt * M, "xi_train", st, &xi_d));
    bool finite = true;
    SCHK(check_xi_finite(ctx, xi_d, (int64_t)nt * M, st, &finite));
    if (!finite) return bail(fail(KLECGC_E_NONFINITE, "xi_train has a non-finite entry"));
    double* Y = nullptr;
    STRY(cudaMalloc(&Y, (size_t)nt * NC * 8));
    struct Guard {
        double* p;
        ~Guard() { cudaFree(p); }
    } gY{Y};
    if (nonlinear(ctx)) {
        double *a = nullptr, *wf = nullptr;
        SCHK(nl_weights(ctx, xi_d, nt, st, &a, &wf));
        bool capped = false;
        SCHK(nl_sequential(ctx, wf, nt, N, ctx->J, ctx->dT / ctx->J, Y, st, &capped));
        if (capped)
            return bail(fail(KLECGC_E_NOT_CONVERGED, "a snapshot's Newton step reached its cap"));
    } else if (ctx->dim == 1) {
        Operators op;
        SCHK(build_operators(ctx, xi_d, nt, N, ctx->J, ctx->dT, 0.5, 1, 0, st, &op));
        WS(double, scr, "seq_scratch", (size_t)nt * nx);
        if (!scr) return bail(KLECGC_E_OUT_OF_MEMORY);
        launch_fine_sequential(nt, N, nx, ctx->J, ctx->dT / ctx->J * pr->forcing, ctx->u0, op.f64,
                               scr, Y, st);
    } else {
        bool capped = false;
        SCHK(sequential_2d(ctx, xi_d, nt, N, ctx->J, Y, st, &capped));
        if (capped)
            return bail(fail(KLECGC_E_NOT_CONVERGED,
                             "a snapshot's fine step reached the Krylov iteration cap"));
    }
    // 3. mean and covariance C = Ytilde Ytilde^T / n_t: the Gram matrix
    //    Ytilde Ytilde^T on the device, its eigenpairs by parallel Jacobi on
    //    the device (eigenvalues of C = those of the Gram matrix / n_t)
    STRY(ctx->alloc_owned(&ctx->ubar, NC));
    launch_mean_center(Y, nt, NC, ctx->ubar, st);
    double* Cd = nullptr;
    STRY(cudaMalloc(&Cd, (size_t)nt * nt * 8));
    Guard gC{Cd};
    launch_gemm<double>(nt, nt, NC, Y, NC, 1, Y, 1, NC, Cd, nt, false, nullptr, st);
    STRY(cudaGetLastError());
    constexpr int kParts = 2048;
    double* Vtd = nullptr;
    const size_t vt_len = ((size_t)nt * nt + 1) & ~(size_t)1;   // keeps rot 16-byte aligned
    STRY(cudaMalloc(&Vtd, (vt_len + (nt / 2 + 1) * 2 + 2 * kParts) * 8 + 64));
    Guard gV{Vtd};
    double2* rot = reinterpret_cast<double2*>(Vtd + vt_len);
    double* part = reinterpret_cast<double*>(rot + nt / 2 + 1);
    int* infod = reinterpret_cast<int*>(part + 2 * kParts);
    // threshold 4 eps ||C||_F: a rotation leaves rounding of about eps |a_pp|
    // in its entry, so entries below it carry no information
    const double jtol = 4 * 2.220446049250313e-16;
    STRY(launch_jacobi_eig(nt, Cd, Vtd, rot, part, kParts, jtol, 100, infod, st));
    std::vector<double> diag(nt);
    int info = 0;
    STRY(cudaMemcpy2DAsync(diag.data(), 8, Cd, (size_t)(nt + 1) * 8, 8, nt,
                           cudaMemcpyDeviceToHost, st));
    STRY(cudaMemcpyAsync(&info, infod, sizeof(int), cudaMemcpyDeviceToHost, st));
    STRY(cudaStreamSynchronize(st));
    if (info < 0) return bail(fail(KLECGC_E_CUDA, "eigensolver did not converge"));
    std::vector<int> order(nt);
    for (int k = 0; k < nt; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return diag[a] > diag[b]; });
    std::vector<double> ev(nt);
    for (int k = 0; k < nt; ++k) ev[k] = diag[order[k]] / nt;
    double total = 0.0;
    for (double e : ev) total += e;
    ctx->lambda_sum = total;
    // M_Q: smallest count with captured fraction >= 1 - eps_kl, at most n_t - 1
    int MQ = nt - 1;
    double acc = 0.0;
    for (int k = 0; k < nt; ++k) {
        acc += ev[k];
        if (acc >= (1.0 - pr->eps_kl) * total) {
            MQ = k + 1;
            break;
        }
    }
    MQ = std::max(1, std::min(MQ, nt - 1));
    while (MQ > 1 && !(ev[MQ - 1] > 0)) --MQ;
    if (!(ev[0] > 0)) return bail(fail(KLECGC_E_INVALID_ARG, "the training snapshots do not vary"));
    ctx->MQ = MQ;
    ctx->lambda_kept = 0.0;
    for (int k = 0; k < MQ; ++k) ctx->lambda_kept += ev[k];
    // 4. modes g_k = (lambda_k n_t)^{-1/2} sum_j e_k^j ytilde_j, and
    //    zeta_k(xi_j) = lambda_k^{-1/2} (ytilde_j, g_k) = sqrt(n_t) e_k^j
    std::vector<double> kept(2 * (size_t)MQ);
    for (int k = 0; k < MQ; ++k) {
        kept[k] = ev[k];
        kept[MQ + k] = std::sqrt(ev[k]);
    }
    double* small = nullptr;   // [MQ] ev, [MQ] sqrt(ev), [MQ] indices
    STRY(cudaMalloc(&small, (2 * (size_t)MQ + MQ) * 8));
    Guard gS{small};
    int* idxd = reinterpret_cast<int*>(small + 2 * MQ);
    STRY(cudaMemcpyAsync(small, kept.data(), kept.size() * 8, cudaMemcpyHostToDevice, st));
    STRY(cudaMemcpyAsync(idxd, order.data(), (size_t)MQ * sizeof(int), cudaMemcpyHostToDevice, st));
    double *Esd = nullptr, *Gd = nullptr;
    STRY(cudaMalloc(&Esd, 2 * (size_t)MQ * nt * 8));
    Guard gE{Esd};
    double* Dcd = Esd + (size_t)MQ * nt;
    launch_gather_modes(Vtd, nt, idxd, small, MQ, Esd, Dcd, st);
    STRY(cudaMalloc(&Gd, (size_t)MQ * NC * 8));
    Guard gG{Gd};
    // G[k][c] = sum_j Es[k][j] Y[j][c]
    launch_gemm<double>(MQ, NC, nt, Esd, nt, 1, Y, NC, 1, Gd, NC, false, nullptr, st);
    // 5. B = psi(Xi_t), least squares H = argmin ||B H - D|| on the device
    //    (Householder QR), H scaled by sqrt(lambda_k) per column
    if (nt < P) return bail(fail(KLECGC_E_INVALID_ARG, "n_train must be >= number of gPC terms"));
    double* Bd = nullptr;
    STRY(cudaMalloc(&Bd, (2 * (size_t)nt * P + nt + (size_t)P * MQ) * 8 + 64));
    Guard gB{Bd};
    double* Bcd = Bd + (size_t)nt * P;
    double* vd = Bcd + (size_t)nt * P;
    double* Hd = vd + nt;
    int* linfo = reinterpret_cast<int*>(Hd + (size_t)P * MQ);
    launch_psi<double>(xi_d, nt, M, ctx->degrees, P, Bd, P, st);
    launch_transpose64(Bd, nt, P, Bcd, st);
    launch_lstsq_qr(nt, P, MQ, Bcd, Dcd, vd, small + MQ, Hd, linfo, st);
    STRY(cudaGetLastError());
    STRY(cudaMemcpyAsync(&info, linfo, sizeof(int), cudaMemcpyDeviceToHost, st));
    STRY(cudaStreamSynchronize(st));
    if (info != 0) return bail(fail(KLECGC_E_INVALID_ARG, "gPC design matrix is rank deficient"));
    // 6. W = (H diag(sqrt(lambda))) G
    STRY(ctx->alloc_owned(&ctx->W, (size_t)P * NC));
    STRY(ctx->alloc_owned(&ctx->W32, (size_t)P * NC));
    ctx->Kp = guess_tc_k_padded(P);
    STRY(ctx->alloc_owned(&ctx->W32t, (size_t)ctx->Kp * NC));
    STRY(ctx->alloc_owned(&ctx->W32t_lo, (size_t)ctx->Kp * NC));
    STRY(ctx->alloc_owned(&ctx->tc_err, 1));
    STRY(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), st));
    launch_gemm<double>(P, NC, MQ, Hd, MQ, 1, Gd, NC, 1, ctx->W, NC, false, nullptr, st);
    launch_to_float(ctx->W, ctx->W32, (int64_t)P * NC, st);
    launch_pad_transpose(ctx->W32, P, NC, ctx->Kp, ctx->W32t, st);
    launch_split_tf32(ctx->W32t, (int64_t)ctx->Kp * NC, ctx->W32t, ctx->W32t_lo, st);
    STRY(ctx->alloc_owned(&ctx->ubar_df, NC));
    STRY(cudaMemcpyAsync(ctx->ubar_df, ctx->ubar, NC * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_to_pairs(reinterpret_cast<double*>(ctx->ubar_df), (int64_t)NC, st);
    STRY(cudaGetLastError());
    STRY(cudaStreamSynchronize(st));
    // release the training-sized scratch
    for (auto& kv : ctx->ws)
        if (kv.second.ptr) cudaFree(kv.second.ptr);
    ctx->ws.clear();
    *out = ctx;
    return KLECGC_OK;
#undef STRY
#undef SCHK
}

klecgc_status klecgc_field(klecgc_ctx* ctx, const double* xi, int64_t S, double* a_out,
                           void* stream) {
    set_error("");
    if (!ctx || !xi || !a_out || S < 0) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double* xi_d = nullptr;
    klecgc_status s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d);
    if (s != KLECGC_OK) return s;
    double* a = nullptr;
    if ((s = build_field(ctx, xi_d, S, st, &a)) != KLECGC_OK) return s;
    TRY(cudaMemcpyAsync(a_out, a, (size_t)S * ctx->nf * 8, cudaMemcpyDefault, st));
    TRY(cudaStreamSynchronize(st));
    return KLECGC_OK;
}

klecgc_status klecgc_guess(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t precision,
                           double* U0_out, void* stream) {
    set_error("");
    if (!ctx || !xi || !U0_out || S < 0 || precision < 0 || precision > 2)
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double* xi_d = nullptr;
    klecgc_status s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d);
    if (s != KLECGC_OK) return s;
    WS(double, U, "U", S * (int64_t)ctx->ns * ctx->N);
    if ((s = gpc_guess_internal(ctx, xi_d, S, precision == KLECGC_FP64, U, st)) != KLECGC_OK)
        return s;
    if ((s = export_batch(ctx, U, S, ctx->N, U0_out, st)) != KLECGC_OK) return s;
    TRY(cudaStreamSynchronize(st));
    return check_tc(ctx, st);
}

klecgc_status klecgc_reference(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N, int32_t J,
                               double* U_out, void* stream) {
    set_error("");
    if (!ctx || !xi || !U_out || S < 0 || N < 1 || J < 1)
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double* xi_d = nullptr;
    klecgc_status s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d);
    if (s != KLECGC_OK) return s;
    const double dT = ctx->prob.T / N;
    WS(double, U, "Uref", S * (int64_t)ctx->ns * N);
    bool capped = false;
    if (nonlinear(ctx)) {
        double *a = nullptr, *wf = nullptr;
        if ((s = nl_weights(ctx, xi_d, S, st, &a, &wf)) != KLECGC_OK) return s;
        if ((s = nl_sequential(ctx, wf, S, N, J, dT / J, U, st, &capped)) != KLECGC_OK) return s;
    } else if (ctx->dim == 2) {
        if ((s = sequential_2d(ctx, xi_d, S, N, J, U, st, &capped)) != KLECGC_OK) return s;
    } else {
        Operators op;
        if ((s = build_operators(ctx, xi_d, S, N, J, dT, 0.5, 1, 0, st, &op)) != KLECGC_OK) return s;
        WS(double, scr, "seq_scratch", S * (int64_t)ctx->nx);
        launch_fine_sequential(S, N, ctx->nx, J, dT / J * ctx->prob.forcing, ctx->u0, op.f64, scr,
                               U, st);
        TRY(cudaGetLastError());
    }
    if ((s = export_batch(ctx, U, S, N, U_out, st)) != KLECGC_OK) return s;
    TRY(cudaStreamSynchronize(st));
    if (capped) return fail(KLECGC_E_NOT_CONVERGED, "a fine step reached its iteration cap");
    return KLECGC_OK;
}

klecgc_status klecgc_mlp_set(klecgc_ctx* ctx, const float* params, int64_t n_params,
                            const float* out_mean, const float* out_std) {
    set_error("");
    if (!ctx || !params) return fail(KLECGC_E_INVALID_ARG, "NULL argument");
    klecgc_status s = mlp_alloc(ctx);
    if (s != KLECGC_OK) return s;
    MlpState& q = ctx->mlp;
    if (n_params != q.P)
        return fail(KLECGC_E_INVALID_ARG, "expected " + std::to_string(q.P) + " parameters");
    TRY(cudaMemcpy(q.theta, params, q.P * 4, cudaMemcpyDefault));
    launch_f32_to_bf16(q.P, q.theta, q.thb, 0);
    std::vector<float> mu(q.D, 0.f), sd(q.D, 1.f);
    if (out_mean) TRY(cudaMemcpy(mu.data(), out_mean, q.D * 4, cudaMemcpyDefault));
    if (out_std) TRY(cudaMemcpy(sd.data(), out_std, q.D * 4, cudaMemcpyDefault));
    std::vector<float> inv(q.D);
    for (int c = 0; c < q.D; ++c) {
        if (!(sd[c] > 0) || !std::isfinite(sd[c]) || !std::isfinite(mu[c]))
            return fail(KLECGC_E_INVALID_ARG, "output normalization must be finite, std > 0");
        inv[c] = 1.f / sd[c];
    }
    TRY(cudaMemcpy(q.mean, mu.data(), q.D * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(q.stdv, sd.data(), q.D * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(q.inv_std, inv.data(), q.D * 4, cudaMemcpyHostToDevice));
    TRY(cudaDeviceSynchronize());
    q.ready = true;
    return KLECGC_OK;
}

klecgc_status klecgc_mlp_get(const klecgc_ctx* ctx, float* params, float* out_mean,
                            float* out_std, int64_t* n_params) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    const MlpState& q = ctx->mlp;
    if (n_params) *n_params = q.theta ? q.P : (int64_t)(ctx->M * 256 + 256 + 2 * (256 * 256 + 256) +
                                                        256 * 64 * ctx->N + 64 * ctx->N);
    if (!q.theta) return params || out_mean || out_std ? fail(KLECGC_E_INVALID_ARG, "no network") : KLECGC_OK;
    if (params) TRY(cudaMemcpy(params, q.theta, q.P * 4, cudaMemcpyDefault));
    if (out_mean) TRY(cudaMemcpy(out_mean, q.mean, q.D * 4, cudaMemcpyDefault));
    if (out_std) TRY(cudaMemcpy(out_std, q.stdv, q.D * 4, cudaMemcpyDefault));
    return KLECGC_OK;
}

klecgc_status klecgc_mlp_loss_grad(klecgc_ctx* ctx, const double* xi, const float* targets,
                                   int64_t B, double* loss_out, float* grad_out, void* stream) {
    set_error("");
    if (!ctx || !xi || !targets || B < 1 || B > (1 << 20)) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (!ctx->mlp.ready) return fail(KLECGC_E_INVALID_ARG, "set the network first (klecgc_mlp_set)");
    cudaStream_t st = (cudaStream_t)stream;
    MlpState& q = ctx->mlp;
    const double* xi_d = nullptr;
    const float* tg = nullptr;
    klecgc_status s = stage_in(ctx, xi, (size_t)B * ctx->M, "mlp_xi", st, &xi_d);
    if (s != KLECGC_OK) return s;
    if ((s = stage_in(ctx, targets, (size_t)B * q.D, "mlp_targets", st, &tg)) != KLECGC_OK) return s;
    MlpBuffers b;
    if ((s = mlp_buffers(ctx, (int)B, &b)) != KLECGC_OK) return s;
    WS(__nv_bfloat16, X, "mlp_X", (size_t)B * q.sizes[0]);
    WS(float, T, "mlp_T", (size_t)B * q.D);
    WS(float, Y, "mlp_Y", (size_t)B * q.D);
    WS(float, dY, "mlp_dY", (size_t)B * q.D);
    WS(__nv_bfloat16, dYb, "mlp_dYb", (size_t)B * q.D);
    WS(float, lsum, "mlp_loss", 1);
    TRY(cudaMemsetAsync(lsum, 0, sizeof(float), st));
    launch_mlp_gather((int)B, q.sizes[0], q.D, nullptr, 0, xi_d, tg, q.mean, q.inv_std, X, T, st);
    {
        const klecgc_status ms_ = mlp_forward(ctx, (int)B, X, b, Y, st);
        if (ms_ != KLECGC_OK) return ms_;
    }
    launch_mse(B * q.D, 1.f / (float)(B * q.D), 1.f / (float)(B * q.D), Y, T, dY, dYb, lsum, st);
    {
        const klecgc_status ms_ = mlp_backward(ctx, (int)B, X, b, dY, dYb, st);
        if (ms_ != KLECGC_OK) return ms_;
    }
    TRY(cudaGetLastError());
    float lh = 0.f;
    TRY(cudaMemcpyAsync(&lh, lsum, sizeof(float), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (loss_out) *loss_out = lh;
    if (grad_out) TRY(cudaMemcpy(grad_out, q.grad, q.P * 4, cudaMemcpyDefault));
    return check_tc(ctx, st);
}

klecgc_status klecgc_mlp_train(klecgc_ctx* ctx, const double* xi, const float* targets, int64_t n,
                               int32_t epochs, int32_t batch, double lr, double lr_final,
                               uint64_t seed, int32_t fit_norm, float* epoch_loss, void* stream) {
    set_error("");
    if (!ctx || !xi || !targets || n < 1 || epochs < 1 || batch < 1 || batch > n || !(lr > 0) ||
        !(lr_final >= 0))
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (!ctx->mlp.ready) return fail(KLECGC_E_INVALID_ARG, "set the initial network first (klecgc_mlp_set)");
    cudaStream_t st = (cudaStream_t)stream;
    MlpState& q = ctx->mlp;
    const double* xi_d = nullptr;
    const float* tg = nullptr;
    klecgc_status s = stage_in(ctx, xi, (size_t)n * ctx->M, "mlp_train_xi", st, &xi_d);
    if (s != KLECGC_OK) return s;
    if ((s = stage_in(ctx, targets, (size_t)n * q.D, "mlp_train_t", st, &tg)) != KLECGC_OK) return s;
    if (fit_norm) launch_colstats(n, q.D, tg, q.mean, q.stdv, q.inv_std, st);
    const int B = batch;
    MlpBuffers b;
    if ((s = mlp_buffers(ctx, B, &b)) != KLECGC_OK) return s;
    WS(__nv_bfloat16, X, "mlp_X", (size_t)B * q.sizes[0]);
    WS(float, T, "mlp_T", (size_t)B * q.D);
    WS(float, Y, "mlp_Y", (size_t)B * q.D);
    WS(float, dY, "mlp_dY", (size_t)B * q.D);
    WS(__nv_bfloat16, dYb, "mlp_dYb", (size_t)B * q.D);
    WS(float, lsum, "mlp_loss", 1);
    WS(int, perm_d, "mlp_perm", (size_t)n);
    TRY(cudaMemsetAsync(q.m, 0, q.P * 4, st));
    TRY(cudaMemsetAsync(q.v, 0, q.P * 4, st));
    q.adam_t = 0;
    const int64_t nb = n / B;
    const double total = (double)epochs * nb;
    std::vector<int> perm(n);
    uint64_t state = seed * 0x9E3779B97F4A7C15ull + 0x2545F4914F6CDD1Dull;
    auto next = [&]() {  // xorshift64*
        state ^= state >> 12;
        state ^= state << 25;
        state ^= state >> 27;
        return state * 0x2545F4914F6CDD1Dull;
    };
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
        for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[next() % (uint64_t)(i + 1)]);
        TRY(cudaMemcpyAsync(perm_d, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        TRY(cudaMemsetAsync(lsum, 0, sizeof(float), st));
        for (int64_t bi = 0; bi < nb; ++bi) {
            q.adam_t += 1;
            const double frac = (q.adam_t - 1) / total;
            const float lr_t = (float)(lr_final + 0.5 * (lr - lr_final) * (1.0 + std::cos(3.14159265358979 * frac)));
            launch_mlp_gather(B, q.sizes[0], q.D, perm_d, (int)(bi * B), xi_d, tg, q.mean,
                              q.inv_std, X, T, st);
            {
                const klecgc_status ms_ = mlp_forward(ctx, B, X, b, Y, st);
                if (ms_ != KLECGC_OK) return ms_;
            }
            const float sc = 1.f / (float)((int64_t)B * q.D);
            launch_mse((int64_t)B * q.D, sc, sc / (float)nb, Y, T, dY, dYb, lsum, st);
            {
                const klecgc_status ms_ = mlp_backward(ctx, B, X, b, dY, dYb, st);
                if (ms_ != KLECGC_OK) return ms_;
            }
            launch_adam(q.P, lr_t, q.adam_t, q.theta, q.grad, q.m, q.v, q.thb, st);
        }
        TRY(cudaGetLastError());
        float lh = 0.f;
        TRY(cudaMemcpyAsync(&lh, lsum, sizeof(float), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (epoch_loss) epoch_loss[ep] = lh;
        if (!std::isfinite(lh)) return fail(KLECGC_E_NONFINITE, "training loss is not finite");
        klecgc_status ts = check_tc(ctx, st);
        if (ts != KLECGC_OK) return ts;
    }
    return KLECGC_OK;
}

klecgc_status klecgc_mlp_guess(klecgc_ctx* ctx, const double* xi, int64_t S, double* U0_out,
                               void* stream) {
    set_error("");
    if (!ctx || !xi || !U0_out || S < 0 || S > (1 << 20)) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (!ctx->mlp.ready) return fail(KLECGC_E_INVALID_ARG, "no network (klecgc_mlp_set / klecgc_mlp_train)");
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double* xi_d = nullptr;
    klecgc_status s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d);
    if (s != KLECGC_OK) return s;
    WS(double, U, "U", S * (int64_t)ctx->nx * ctx->N);
    bool finite = true;
    if ((s = mlp_guess_internal(ctx, xi_d, S, U, st, &finite)) != KLECGC_OK) return s;
    if ((s = export_batch(ctx, U, S, ctx->N, U0_out, st)) != KLECGC_OK) return s;
    TRY(cudaStreamSynchronize(st));
    if ((s = check_tc(ctx, st)) != KLECGC_OK) return s;
    return finite ? KLECGC_OK : fail(KLECGC_E_NONFINITE, "network output is not finite");
}

klecgc_status klecgc_downsample(klecgc_ctx* ctx, const double* U, int64_t S, int32_t N,
                                float* T_out, void* stream) {
    set_error("");
    if (!ctx || !U || !T_out || S < 0 || N < 1) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (ctx->dim != 1) return fail(KLECGC_E_UNSUPPORTED, "the network grid is 1D only");
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const double* Ud = nullptr;
    klecgc_status s = stage_in(ctx, U, (size_t)S * N * ctx->nx, "ds_in", st, &Ud);
    if (s != KLECGC_OK) return s;
    float* T = T_out;
    const bool dev = is_device_ptr(T_out);
    if (!dev) {
        WS(float, t, "ds_out", (size_t)S * N * 64);
        T = t;
    }
    launch_downsample(S * (int64_t)N, ctx->nx, Ud, T, st);
    TRY(cudaGetLastError());
    if (!dev) TRY(cudaMemcpyAsync(T_out, T, (size_t)S * N * 64 * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    return KLECGC_OK;
}

klecgc_status klecgc_mlp_set_residual(klecgc_ctx* ctx, int32_t residual) {
    set_error("");
    if (!ctx || residual < 0 || residual > 1) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (ctx->dim != 1 || nonlinear(ctx))
        return fail(KLECGC_E_UNSUPPORTED, "the learned guess is for the linear 1D problem only");
    ctx->mlp.residual = residual != 0;
    return KLECGC_OK;
}

klecgc_status klecgc_mlp_targets(klecgc_ctx* ctx, const double* xi, const double* U, int64_t S,
                                 float* T_out, void* stream) {
    set_error("");
    if (!ctx || !xi || !U || !T_out || S < 0) return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (ctx->dim != 1 || nonlinear(ctx))
        return fail(KLECGC_E_UNSUPPORTED, "the learned guess is for the linear 1D problem only");
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = ctx->N;
    const double* Ud = nullptr;
    klecgc_status s = stage_in(ctx, U, (size_t)S * N * ctx->nx, "ds_in", st, &Ud);
    if (s != KLECGC_OK) return s;
    float* T = T_out;
    const bool dev = is_device_ptr(T_out);
    if (!dev) {
        WS(float, t, "ds_out", (size_t)S * N * 64);
        T = t;
    }
    launch_downsample(S * (int64_t)N, ctx->nx, Ud, T, st);
    if (ctx->mlp.residual) {
        const double* xi_d = nullptr;
        if ((s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d)) != KLECGC_OK) return s;
        WS(double, Ug, "U", S * (int64_t)ctx->nx * N);
        WS(double, Uc, "mlp_gpc", S * (int64_t)ctx->nx * N);
        WS(float, Tg, "mlp_gpc_ds", (size_t)S * N * 64);
        if ((s = gpc_guess_internal(ctx, xi_d, S, false, Ug, st)) != KLECGC_OK) return s;
        if ((s = export_batch(ctx, Ug, S, N, Uc, st)) != KLECGC_OK) return s;
        launch_downsample(S * (int64_t)N, ctx->nx, Uc, Tg, st);
        launch_sub_f32((int64_t)S * N * 64, T, Tg, st);
    }
    TRY(cudaGetLastError());
    if (!dev) TRY(cudaMemcpyAsync(T_out, T, (size_t)S * N * 64 * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    return KLECGC_OK;
}

klecgc_status klecgc_fine_sweep(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N,
                                const double* U_in, double dT, int32_t J, double alpha,
                                int32_t precision, double* r_out, void* stream) {
    set_error("");
    if (!ctx || !xi || !U_in || !r_out || S < 0 || J < 1 || !(alpha > 0 && alpha < 1) ||
        precision < 0 || precision > 2)
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (!pow2_in_range(N)) return fail(KLECGC_E_UNSUPPORTED, "N must be a power of 2 in [2, 64]");
    if (nonlinear(ctx))
        return fail(KLECGC_E_UNSUPPORTED, "stage entry points: linear problems only");
    klecgc_status s = check_dT(ctx, N, dT);
    if (s != KLECGC_OK || S == 0) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = ctx->ns;
    const double* xi_d = nullptr;
    if ((s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d)) != KLECGC_OK) return s;
    if (ctx->dim == 2) {
        if (precision == KLECGC_MIXED_DEFECT)
            return fail(KLECGC_E_UNSUPPORTED, "2D: FP64 or MIXED only");
        if (ctx->prob.advection > 0 && precision != KLECGC_FP64)
            return fail(KLECGC_E_UNSUPPORTED, "advection-diffusion: FP64 only");
        double* wdt = nullptr;
        if ((s = build_weights_2d(ctx, xi_d, S, dT / J, dT, st, &wdt, nullptr)) != KLECGC_OK) return s;
        WS(double, U, "U", S * (int64_t)nx * N);
        if ((s = import_batch(ctx, U_in, S, N, U, st)) != KLECGC_OK) return s;
        WS(double, r, "r", S * (int64_t)nx * N);
        WS(int, active, "active", S);
        TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
        const double dt = dT / J;
        if (use_band(ctx, precision == KLECGC_FP64)) {
            double* Bf = nullptr;
            if ((s = band_factors_fine(ctx, wdt, S, dt, st, &Bf)) != KLECGC_OK) return s;
            WS(double, xs, "band_xN", S * (int64_t)nx * N);
            ctx->launch(KLECGC_K_FINE, st, [&] {
                launch_band_fine(S, N, ctx->nx, J, dt * ctx->prob.reaction, dt * ctx->prob.forcing,
                                 dt * ctx->prob.advection, alpha, 0, U, ctx->u0, wdt, Bf, xs, r,
                                 active, st);
            });
            TRY(cudaGetLastError());
            ctx->kry_it_fine = ctx->kry_it_cgc = 0;
            return export_batch(ctx, r, S, N, r_out, st);
        }
        int* ifail = nullptr;
        unsigned long long* its = nullptr;
        if ((s = krylov_flags(ctx, S, st, &ifail, &its)) != KLECGC_OK) return s;
        const bool mixed = precision == KLECGC_MIXED;
        const Plan2D pl = plan_2d(fine_kind(ctx, mixed), ctx->nx, S * N, ctx->method2d == 3);
        WS(double, scr, "k2d_scratch", pl.scratch_doubles);
        ctx->launch(KLECGC_K_FINE, st, [&] {
            if (mixed)
                launch_fine2d_mixed(pl, S, N, ctx->nx, J, dt * ctx->prob.reaction,
                                    dt * ctx->prob.forcing, alpha, 0, U, ctx->u0, wdt,
                                    ctx->kry_rtol_fine, kInnerRtol, ctx->kry_maxit, r, active,
                                    ifail, its, scr, st);
            else
                launch_fine2d(pl, S, N, ctx->nx, J, dt * ctx->prob.reaction,
                              dt * ctx->prob.forcing, dt * ctx->prob.advection, alpha, 0, U,
                              ctx->u0, wdt, ctx->kry_rtol_fine, ctx->kry_maxit, r, active, ifail,
                              its, scr, st);
        });
        TRY(cudaGetLastError());
        if ((s = export_batch(ctx, r, S, N, r_out, st)) != KLECGC_OK) return s;
        std::vector<int> hf;
        bool capped = false;
        if ((s = krylov_read(ctx, S, ifail, its, st, &hf, &capped)) != KLECGC_OK) return s;
        if (capped) return fail(KLECGC_E_NOT_CONVERGED, "a fine step reached the Krylov iteration cap");
        return KLECGC_OK;
    }
    Operators op;
    if ((s = build_operators(ctx, xi_d, S, N, J, dT, alpha, precision == KLECGC_FP64 ? 1 : 2, 0,
                             st, &op)) != KLECGC_OK)
        return s;
    WS(double, U, "U", S * (int64_t)nx * N);
    if ((s = import_batch(ctx, U_in, S, N, U, st)) != KLECGC_OK) return s;
    WS(double, r, "r", S * (int64_t)nx * N);
    WS(int, active, "active", S);
    TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
    if (precision == KLECGC_FP64) {
        launch_fine_sweep_fp64(S, N, nx, J, dT, alpha, ctx->prob.reaction, ctx->prob.forcing, U,
                               ctx->u0, op.f64, op.wT, r, active, st);
    } else {
        WS(float, fo, "fout", S * (int64_t)nx * N);
        launch_fine_any(op.sh32, S, N, nx, J, dT / J, ctx->prob.reaction, ctx->prob.forcing, 0, U,
                        nullptr, ctx->u0, nullptr, op.tab32, fo, active, st);
        launch_jump_from_f32(S, N, nx, alpha, dT * ctx->prob.reaction, fo, U, op.wT, r, st);
    }
    TRY(cudaGetLastError());
    if ((s = export_batch(ctx, r, S, N, r_out, st)) != KLECGC_OK) return s;
    TRY(cudaStreamSynchronize(st));
    return KLECGC_OK;
}

klecgc_status klecgc_cgc_apply(klecgc_ctx* ctx, const double* xi, int64_t S, int32_t N,
                               const double* r_in, double dT, double alpha, int32_t precision,
                               double* u_out, void* stream) {
    set_error("");
    if (!ctx || !xi || !r_in || !u_out || S < 0 || !(alpha > 0 && alpha < 1) || precision < 0 ||
        precision > 2)
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (ctx->dim == 1 && precision == KLECGC_MIXED)
        return fail(KLECGC_E_INVALID_ARG, "1D: precision FP64 or MIXED_DEFECT");
    if (nonlinear(ctx))
        return fail(KLECGC_E_UNSUPPORTED, "stage entry points: linear problems only");
    if (!pow2_in_range(N)) return fail(KLECGC_E_UNSUPPORTED, "N must be a power of 2 in [2, 64]");
    klecgc_status s = check_dT(ctx, N, dT);
    if (s != KLECGC_OK || S == 0) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = ctx->ns, K = N / 2 + 1;
    const double* xi_d = nullptr;
    if ((s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d)) != KLECGC_OK) return s;
    const bool f64 = precision == KLECGC_FP64;
    if (ctx->dim == 2) {
        if (precision == KLECGC_MIXED_DEFECT)
            return fail(KLECGC_E_UNSUPPORTED, "2D: FP64 or MIXED only");
        if (ctx->prob.advection > 0 && precision != KLECGC_FP64)
            return fail(KLECGC_E_UNSUPPORTED, "advection-diffusion: FP64 only");
        const bool mixed = precision == KLECGC_MIXED;
        double* wdT = nullptr;
        if ((s = build_weights_2d(ctx, xi_d, S, dT, dT, st, nullptr, &wdT)) != KLECGC_OK) return s;
        std::vector<double2> lam;
        double2* lam_d = nullptr;
        if ((s = upload_lambda(ctx, N, alpha, st, lam, &lam_d)) != KLECGC_OK) return s;
        WS(double, r, "r", S * (int64_t)nx * N);
        if ((s = import_batch(ctx, r_in, S, N, r, st)) != KLECGC_OK) return s;
        WS(double, U, "U", S * (int64_t)nx * N);
        WS(int, active, "active", S);
        TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
        double *sc, *isc;
        if ((s = scale_tables<double>(ctx, N, alpha, st, &sc, &isc)) != KLECGC_OK) return s;
        WS(Cplx<double>, p, "p64", S * (int64_t)nx * K);
        if (use_band(ctx, !mixed)) {
            double2* Bc = nullptr;
            if ((s = band_factors_cgc(ctx, wdT, S, K, dT, lam_d, st, &Bc)) != KLECGC_OK) return s;
            launch_cgc_forward<double, double>(S, N, nx, r, sc, p, active, st);
            ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] { launch_band_cgc(S, K, ctx->nx, Bc, p, active, st); });
            launch_cgc_inverse<double>(S, N, nx, p, isc, U, 2, nullptr, nullptr, active, st);
            TRY(cudaGetLastError());
            ctx->kry_it_fine = ctx->kry_it_cgc = 0;
            return export_batch(ctx, U, S, N, u_out, st);
        }
        int* ifail = nullptr;
        unsigned long long* its = nullptr;
        if ((s = krylov_flags(ctx, S, st, &ifail, &its)) != KLECGC_OK) return s;
        const Plan2D pl = plan_2d(cgc_kind(ctx, mixed), ctx->nx, S * K, ctx->method2d == 3);
        WS(double, scr, "k2d_scratch_c", pl.scratch_doubles);
        launch_cgc_forward<double, double>(S, N, nx, r, sc, p, active, st);
        if (mixed)
            launch_cgc_solve2d_mixed(pl, S, K, ctx->nx, dT * ctx->prob.reaction, lam_d, wdT,
                                     ctx->kry_rtol_cgc, kInnerRtol, ctx->kry_maxit, p, active,
                                     ifail, its + 1, scr, st);
        else
            launch_cgc_solve2d(pl, S, K, ctx->nx, dT * ctx->prob.reaction,
                               dT * ctx->prob.advection, lam_d, wdT, ctx->kry_rtol_cgc,
                               ctx->kry_maxit, p, active, ifail, its + 1, scr, st);
        launch_cgc_inverse<double>(S, N, nx, p, isc, U, 2, nullptr, nullptr, active, st);
        TRY(cudaGetLastError());
        if ((s = export_batch(ctx, U, S, N, u_out, st)) != KLECGC_OK) return s;
        std::vector<int> hf;
        bool capped = false;
        if ((s = krylov_read(ctx, S, ifail, its, st, &hf, &capped)) != KLECGC_OK) return s;
        if (capped) return fail(KLECGC_E_NOT_CONVERGED, "a shifted solve reached the Krylov iteration cap");
        return KLECGC_OK;
    }
    Operators op;
    if ((s = build_operators(ctx, xi_d, S, N, 1, dT, alpha, 0, f64 ? 1 : 2, st, &op)) != KLECGC_OK)
        return s;
    WS(double, r, "r", S * (int64_t)nx * N);
    if ((s = import_batch(ctx, r_in, S, N, r, st)) != KLECGC_OK) return s;
    WS(double, U, "U", S * (int64_t)nx * N);
    WS(int, active, "active", S);
    TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
    if (f64) {
        double *sc, *isc;
        if ((s = scale_tables<double>(ctx, N, alpha, st, &sc, &isc)) != KLECGC_OK) return s;
        WS(Cplx<double>, p, "p64", S * (int64_t)nx * K);
        launch_cgc_forward<double, double>(S, N, nx, r, sc, p, active, st);
        launch_cgc_solve<double, double>(S, K, nx, op.dinv64, op.lu64, op.wT, p, active, st);
        launch_cgc_inverse<double>(S, N, nx, p, isc, U, 2, nullptr, nullptr, active, st);
    } else {
        float *sc, *isc;
        if ((s = scale_tables<float>(ctx, N, alpha, st, &sc, &isc)) != KLECGC_OK) return s;
        WS(float, r32, "d32", S * (int64_t)nx * N);
        launch_to_float(r, r32, S * (int64_t)nx * N, st);
        WS(Cplx<float>, p, "p32", S * (int64_t)nx * K);
        launch_cgc_forward<float, float>(S, N, nx, r32, sc, p, active, st);
        launch_cgc_solve<float, float>(S, K, nx, op.dinv32, op.lu32, op.wT32, p, active, st);
        launch_cgc_inverse<float>(S, N, nx, p, isc, U, 2, nullptr, nullptr, active, st);
    }
    TRY(cudaGetLastError());
    if ((s = export_batch(ctx, U, S, N, u_out, st)) != KLECGC_OK) return s;
    TRY(cudaStreamSynchronize(st));
    return KLECGC_OK;
}

}  // extern "C"

namespace {

struct PinnedInts {
    int* p = nullptr;
    ~PinnedInts() {
        if (p) cudaFreeHost(p);
    }
};

// Runs parareal iterations k0, k0 + 1, ... until no sample is active or kmax
// iterations have run (Algorithms 1 and 2: the loop of Step 3).
// iterate(stream, k, kdev) launches one iteration that ends with the stopping
// rule counting the active samples into n_active; with kdev == nullptr the
// iteration number is the host's k, otherwise it is *kdev on the device.
// Loop mode 0 runs the iterations as a CUDA graph whose WHILE node repeats
// the captured iteration while k_loop_tail finds active samples and k < kmax,
// with no host round trip per iteration; loop mode 1, and CUDA-event timing
// of the kernel classes (per-launch events cannot sit in a graph loop), run
// them from the host with a readback of n_active after each.  The iteration
// is captured once, on a private stream, and only launches kernels and
// memsets.  If the graph cannot be built (before anything of it was
// launched), the host loop runs instead.
template <class It>
klecgc_status iterate_loop(klecgc_ctx* ctx, cudaStream_t st, int* kdev, int* n_active, int k0,
                           int kmax, It&& iterate) {
    if (k0 >= kmax) return KLECGC_OK;
    klecgc_status s;
    if (ctx->loop_mode == 0 && !ctx->prof_timing) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        cudaStream_t cs = nullptr;
        bool built = false;
        s = KLECGC_OK;
        do {
            if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) break;
            if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
                break;
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) != cudaSuccess) break;
            cudaGraph_t body = np.conditional.phGraph_out[0];
            if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                break;
            s = iterate(cs, k0, (const int*)kdev);
            launch_loop_tail(kdev, n_active, kmax, h, cs);
            cudaGraph_t captured = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(cs, &captured);
            if (s != KLECGC_OK || ec != cudaSuccess) break;
            if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) break;
            built = true;
        } while (false);
        if (built) {
            launch_set_int(kdev, k0, st);
            cudaError_t e = cudaGraphLaunch(ex, st);
            cudaGraphExecDestroy(ex);   // released once the launch completes
            cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) return fail(KLECGC_E_CUDA, cudaGetErrorString(e));
            TRY(cudaGetLastError());
            return KLECGC_OK;
        }
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        if (cs) cudaStreamDestroy(cs);
        if (s != KLECGC_OK) return s;
        cudaGetLastError();   // graph not available: the host loop below
    }
    PinnedInts pin;
    TRY(cudaMallocHost(&pin.p, sizeof(int)));
    for (int k = k0; k < kmax; ++k) {
        if ((s = iterate(st, k, (const int*)nullptr)) != KLECGC_OK) return s;
        TRY(cudaGetLastError());
        TRY(cudaMemcpyAsync(pin.p, n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        TRY(cudaStreamSynchronize(st));
        if (*pin.p == 0) break;
    }
    return KLECGC_OK;
}

// Scratch names carry `tag` while a run's code executes.
struct TagScope {
    klecgc_ctx* ctx;
    std::string saved;
    TagScope(klecgc_ctx* c, const std::string& t) : ctx(c), saved(c->ws_tag) { c->ws_tag = t; }
    ~TagScope() { ctx->ws_tag = saved; }
};

// One solve of S samples with one context and one (N, J, dT): the online
// part of Algorithm 3 split into begin (operators, guess), step (one
// parareal iteration: F, the CGC steps (a)-(c), the stopping rule, and an
// asynchronous copy of the active count) and finish (export).  klecgc_solve
// runs one; klecgc_solve_batch interleaves several, one per class of equal
// (context, J), on a pool of streams.
struct SolveRun {
    klecgc_ctx* ctx = nullptr;
    std::string tag;
    cudaStream_t st = nullptr;
    int64_t S = 0;
    int N = 0, J = 0, K = 0, nx = 0, kmax = 0, precision = 0, guess = 0;
    double dT = 0, alpha = 0, tol = 0;
    bool f64 = false, defect = false;
    Operators op;
    double *wdt2 = nullptr, *wdT2 = nullptr;  // 2D face weights (fine, CGC)
    double* U = nullptr;
    int* active = nullptr;
    int32_t *iters = nullptr, *status = nullptr;
    unsigned long long* delta = nullptr;
    int* n_active = nullptr;
    double *sc64 = nullptr, *isc64 = nullptr;
    float *sc32 = nullptr, *isc32 = nullptr;
    double* r = nullptr;                       // FP64 path: CGC right-hand side
    Cplx<double>* p64 = nullptr;
    Cplx<float>* p32 = nullptr;
    float* fout = nullptr;                     // mixed paths: FP32 fine result
    float* c32 = nullptr;                      // mixed paths: FP32 increment of U
    float2* Facc2[2] = {nullptr, nullptr};     // defect: F(U_{n-1}) as pairs, two buffers
    float2* Udf = nullptr;                     // defect: the iterate as pairs (aliases U)
    int* ifail = nullptr;                      // 2D: Krylov cap flags and counters
    unsigned long long* kits = nullptr;
    double2* lam_d = nullptr;
    Plan2D plF, plC;
    bool band = false;                         // 2D: banded LU instead of Krylov
    double* Bf = nullptr;                      // band factors of the fine step
    double2* Bc = nullptr;                     // band factors of the shifted systems
    double* xband = nullptr;                   // band: fine-sweep vectors
    double *scrF = nullptr, *scrC = nullptr;
    int* h_active = nullptr;                   // pinned, one int (owned by the caller)
    int k_next = 0;

    int* kdev = nullptr;                       // device iteration counter (graph loop)

    klecgc_status begin(const double* xi_d, const double* U_guess);
    // one parareal iteration on stream `s`: the host's k, or *kdev when kdev
    // is given (k then only tells k >= 1 from the first iteration)
    klecgc_status iterate(cudaStream_t s, int k, const int* kd);
    // host-driven: iteration k_next on st, active count copied to *h_active
    klecgc_status step();
    bool finished() const { return *h_active == 0 || k_next >= kmax; }
    klecgc_status finish(double* U_out, std::vector<int32_t>& hs, std::vector<int32_t>& hi,
                         bool* capped);
};

klecgc_status SolveRun::begin(const double* xi_d, const double* U_guess) {
    TagScope ts(ctx, tag);
    klecgc_status s;
    nx = ctx->ns;  // unknowns per time level
    K = N / 2 + 1;
    f64 = precision == KLECGC_FP64;
    defect = precision == KLECGC_MIXED_DEFECT;
    const int64_t NS = S * (int64_t)nx * N;
    if (ctx->dim == 2) {
        if ((s = build_weights_2d(ctx, xi_d, S, dT / J, dT, st, &wdt2, &wdT2)) != KLECGC_OK) return s;
    } else if ((s = build_operators(ctx, xi_d, S, N, J, dT, alpha, f64 ? 1 : 2, defect ? 2 : 1, st,
                                    &op)) != KLECGC_OK) {
        return s;
    }
    {
        WS(double, u, "U", NS);
        U = u;
    }
    bool mlp_ok = false;
    if (guess == KLECGC_GUESS_MLP) {
        if ((s = mlp_guess_internal(ctx, xi_d, S, U, st, &mlp_ok)) != KLECGC_OK) return s;
    }
    // the defect path keeps U as FP32 pairs; the tensor-core guess writes them
    // directly (1D)
    const bool guess_pairs = defect && ctx->dim == 1 && guess == KLECGC_GUESS_GPC;
    if (guess == KLECGC_GUESS_GPC || (guess == KLECGC_GUESS_MLP && !mlp_ok)) {
        // the surrogate is also the fallback of the learned guess (non-finite output)
        if ((s = gpc_guess_internal(ctx, xi_d, S, f64, U, st, guess_pairs)) != KLECGC_OK)
            return s;
    } else if (guess == KLECGC_GUESS_MLP) {
    } else if (guess == KLECGC_GUESS_ZERO) {
        TRY(cudaMemsetAsync(U, 0, NS * sizeof(double), st));
    } else if (guess == KLECGC_GUESS_COARSE) {
        if ((s = coarse_guess_internal(ctx, S, N, dT, ctx->dim == 2 ? wdT2 : op.a, U, st)) != KLECGC_OK)
            return s;
    } else {
        if ((s = import_batch(ctx, U_guess, S, N, U, st)) != KLECGC_OK) return s;
    }
    {
        WS(int, a, "active", S);
        WS(int32_t, it, "iters", S);
        WS(int32_t, sta, "status", S);
        WS(unsigned long long, de, "delta", S);
        WS(int, na, "n_active", 1);
        WS(int, kd, "kdev", 1);
        active = a;
        iters = it;
        status = sta;
        delta = de;
        n_active = na;
        kdev = kd;
    }
    TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
    TRY(cudaMemsetAsync(iters, 0xff, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(status, 0, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(delta, 0, S * sizeof(unsigned long long), st));
    if (defect || (!f64 && ctx->dim == 1)) {
        if ((s = scale_tables<float>(ctx, N, alpha, st, &sc32, &isc32)) != KLECGC_OK) return s;
    }
    if (!defect) {
        if ((s = scale_tables<double>(ctx, N, alpha, st, &sc64, &isc64)) != KLECGC_OK) return s;
    }
    if (!defect) {
        // FP64 path: the CGC right-hand side; mixed path (1D): its scaled
        // FP64 accumulation
        WS(double, rr, "r", NS);
        r = rr;
    }
    if (!defect) {
        WS(Cplx<double>, pp, "p64", S * (int64_t)nx * K);
        p64 = pp;
    } else {
        WS(Cplx<float>, pp, "p32", S * (int64_t)nx * K);
        p32 = pp;
    }
    if (!f64 && ctx->dim == 1) {
        WS(float, fo, "fout", NS);
        WS(float, cc, "c32", NS);
        fout = fo;
        c32 = cc;
        if (defect) {
            WS(float2, fa, "FaccA2", NS);
            WS(float2, fb, "FaccB2", NS);
            Facc2[0] = fa;
            Facc2[1] = fb;
            if (!guess_pairs)
                ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_to_pairs(U, NS, st); });
            Udf = reinterpret_cast<float2*>(U);
        }
    }
    if (ctx->dim == 2) {
        // Krylov solves, or banded LU factors (FP64 on small grids)
        if ((s = krylov_flags(ctx, S, st, &ifail, &kits)) != KLECGC_OK) return s;
        std::vector<double2> lam;
        if ((s = upload_lambda(ctx, N, alpha, st, lam, &lam_d)) != KLECGC_OK) return s;
        band = use_band(ctx, f64);
        if (band) {
            if ((s = band_factors_fine(ctx, wdt2, S, dT / J, st, &Bf)) != KLECGC_OK) return s;
            if ((s = band_factors_cgc(ctx, wdT2, S, K, dT, lam_d, st, &Bc)) != KLECGC_OK) return s;
            WS(double, xb, "band_xN", S * (int64_t)nx * N);
            xband = xb;
            TRY(cudaGetLastError());
            k_next = 0;
            *h_active = 1;
            return KLECGC_OK;
        }
        plF = plan_2d(fine_kind(ctx, precision == KLECGC_MIXED), ctx->nx, S * N, ctx->method2d == 3);
        plC = plan_2d(cgc_kind(ctx, precision == KLECGC_MIXED), ctx->nx, S * K, ctx->method2d == 3);
        WS(double, a1, "k2d_scratch", plF.scratch_doubles);
        WS(double, a2, "k2d_scratch_c", plC.scratch_doubles);
        scrF = a1;
        scrC = a2;
    }
    TRY(cudaGetLastError());
    k_next = 0;
    *h_active = 1;
    return KLECGC_OK;
}

klecgc_status SolveRun::step() {
    klecgc_status s = iterate(st, k_next++, nullptr);
    if (s != KLECGC_OK) return s;
    TRY(cudaMemcpyAsync(h_active, n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    return KLECGC_OK;
}

klecgc_status SolveRun::iterate(cudaStream_t st, int k, const int* kd) {
    TagScope ts(ctx, tag);
    const double dTreact = dT * ctx->prob.reaction;
    if (ctx->dim == 2 && band) {
        const double dt = dT / J;
        ctx->launch(KLECGC_K_FINE, st, [&] {
            launch_band_fine(S, N, ctx->nx, J, dt * ctx->prob.reaction, dt * ctx->prob.forcing,
                             dt * ctx->prob.advection, alpha, 0, U, ctx->u0, wdt2, Bf, xband, r,
                             active, st);
        });
        ctx->launch(KLECGC_K_CGC_FWD, st, [&] { launch_cgc_forward<double, double>(S, N, nx, r, sc64, p64, active, st); });
        ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] { launch_band_cgc(S, K, ctx->nx, Bc, p64, active, st); });
        ctx->launch(KLECGC_K_CGC_INV, st, [&] { launch_cgc_inverse<double>(S, N, nx, p64, isc64, U, 0, delta, nullptr, active, st); });
    } else if (ctx->dim == 2) {
        const double dt = dT / J;
        if (precision == KLECGC_MIXED)
            ctx->launch(KLECGC_K_FINE, st, [&] {
                launch_fine2d_mixed(plF, S, N, ctx->nx, J, dt * ctx->prob.reaction,
                                    dt * ctx->prob.forcing, alpha, 0, U, ctx->u0, wdt2,
                                    ctx->kry_rtol_fine, kInnerRtol, ctx->kry_maxit, r, active,
                                    ifail, kits, scrF, st);
            });
        else
            ctx->launch(KLECGC_K_FINE, st, [&] {
                launch_fine2d(plF, S, N, ctx->nx, J, dt * ctx->prob.reaction,
                              dt * ctx->prob.forcing, dt * ctx->prob.advection, alpha, 0, U,
                              ctx->u0, wdt2, ctx->kry_rtol_fine, ctx->kry_maxit, r, active,
                              ifail, kits, scrF, st);
            });
        ctx->launch(KLECGC_K_CGC_FWD, st, [&] { launch_cgc_forward<double, double>(S, N, nx, r, sc64, p64, active, st); });
        ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] {
            if (precision == KLECGC_MIXED)
                launch_cgc_solve2d_mixed(plC, S, K, ctx->nx, dTreact, lam_d, wdT2,
                                         ctx->kry_rtol_cgc, kInnerRtol, ctx->kry_maxit, p64,
                                         active, ifail, kits + 1, scrC, st);
            else
                launch_cgc_solve2d(plC, S, K, ctx->nx, dTreact, dT * ctx->prob.advection, lam_d,
                                   wdT2, ctx->kry_rtol_cgc, ctx->kry_maxit, p64, active, ifail,
                                   kits + 1, scrC, st);
        });
        ctx->launch(KLECGC_K_CGC_INV, st, [&] { launch_cgc_inverse<double>(S, N, nx, p64, isc64, U, 0, delta, nullptr, active, st); });
    } else {
        if (f64) {
            ctx->launch(KLECGC_K_FINE, st, [&] {
                launch_fine_sweep_fp64(S, N, nx, J, dT, alpha, ctx->prob.reaction,
                                       ctx->prob.forcing, U, ctx->u0, op.f64, op.wT, r, active, st);
            });
            ctx->launch(KLECGC_K_CGC_FWD, st, [&] { launch_cgc_forward<double, double>(S, N, nx, r, sc64, p64, active, st); });
        } else {
            // F(start) on the first iteration, F0(increment) afterwards
            ctx->launch(KLECGC_K_FINE, st, [&] {
                launch_fine_any(op.sh32, S, N, nx, J, dT / J, ctx->prob.reaction, ctx->prob.forcing,
                              k == 0 ? 0 : 1, defect ? nullptr : U, Udf, ctx->u0, c32, op.tab32,
                              fout, active, st);
            });
            if (defect)
                ctx->launch(KLECGC_K_CGC_FWD, st, [&] {
                    launch_cgc_forward_df(S, N, nx, fout, Facc2[0], Facc2[1], k, kd, Udf, op.wT,
                                          dTreact, sc32, p32, active, st);
                });
            else
                ctx->launch(KLECGC_K_CGC_FWD, st, [&] {
                    launch_cgc_forward_acc(S, N, nx, fout, k == 0 ? nullptr : c32, U, op.wT,
                                           dTreact, alpha, sc64, sc32, r, p64, active, st);
                });
        }
        if (!defect) {
            ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] { launch_cgc_solve<double, double>(S, K, nx, op.dinv64, op.lu64, op.wT, p64, active, st); });
            ctx->launch(KLECGC_K_CGC_INV, st, [&] { launch_cgc_inverse<double>(S, N, nx, p64, isc64, U, 0, delta, c32, active, st); });
        } else {
            ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] { launch_cgc_solve<float, float>(S, K, nx, op.dinv32, op.lu32, op.wT32, p32, active, st); });
            ctx->launch(KLECGC_K_CGC_INV, st, [&] { launch_cgc_inverse_df(S, N, nx, p32, isc32, Udf, delta, c32, active, st); });
        }
    }
    TRY(cudaMemsetAsync(n_active, 0, sizeof(int), st));
    ctx->launch(KLECGC_K_CONV, st, [&] { launch_convergence(S, k, kmax, tol, delta, active, iters, status, n_active, st, kd); });
    TRY(cudaGetLastError());
    return KLECGC_OK;
}

// U_out: [S][N][n] (host or device).  hs / hi receive the per-sample status
// and iteration counts (the stream is synchronized).
klecgc_status SolveRun::finish(double* U_out, std::vector<int32_t>& hs, std::vector<int32_t>& hi,
                               bool* capped) {
    TagScope ts(ctx, tag);
    klecgc_status s;
    const int64_t NS = S * (int64_t)nx * N;
    if (defect) {
        // pairs -> FP64 in the caller's layout
        if (is_device_ptr(U_out)) {
            ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_pairs_transpose_out(Udf, U_out, S, nx, N, st); });
        } else {
            WS(double, tmp, "export", NS);
            ctx->launch(KLECGC_K_LAYOUT, st, [&] { launch_pairs_transpose_out(Udf, tmp, S, nx, N, st); });
            TRY(cudaMemcpyAsync(U_out, tmp, NS * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        TRY(cudaGetLastError());
    } else if ((s = export_batch(ctx, U, S, N, U_out, st)) != KLECGC_OK) {
        return s;
    }
    hs.assign(S, 0);
    hi.assign(S, 0);
    TRY(cudaMemcpyAsync(hs.data(), status, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hi.data(), iters, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if ((s = check_tc(ctx, st)) != KLECGC_OK) return s;
    *capped = false;
    if (ctx->dim == 2) {
        // a sample whose Krylov solve reached the cap has an inexact iterate
        std::vector<int> hf;
        if ((s = krylov_read(ctx, S, ifail, kits, st, &hf, capped)) != KLECGC_OK) return s;
        for (int64_t i = 0; i < S; ++i)
            if (hf[i] && hs[i] == KLECGC_OK) hs[i] = KLECGC_E_NOT_CONVERGED;
    }
    return KLECGC_OK;
}

// The uneven batch with every class advancing together (Algorithm 2 for all
// instances at once): each parareal iteration is one persistent launch per
// stage over all classes (the fine stage one per rows-per-lane group), whose
// CTAs pull (class, sample, part) tasks from a work queue ordered longest
// first; the iterations run as a CUDA graph WHILE loop (iterate_loop).  The
// classes were set up by SolveRun::begin on the pool streams.
klecgc_status batch_persistent(klecgc_ctx* c0, std::vector<SolveRun>& runs, int64_t n, int kmax,
                               double tol, cudaStream_t st, const std::vector<cudaStream_t>& pool) {
    klecgc_ctx* ctx = c0;
    const int nc = (int)runs.size();
    const int defect = runs[0].defect ? 1 : 0;
    // order after the set-up on the pool streams
    {
        cudaEvent_t ev;
        TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        for (cudaStream_t x : pool) {
            cudaEventRecord(ev, x);
            cudaStreamWaitEvent(st, ev, 0);
        }
        cudaEventDestroy(ev);
    }
    std::vector<BatchClass> hc(nc);
    for (int c = 0; c < nc; ++c) {
        SolveRun& R = runs[c];
        klecgc_ctx* x = R.ctx;
        BatchClass& C = hc[c];
        C = BatchClass{};
        C.S = R.S;
        C.nx = R.nx;
        C.N = R.N;
        C.K = R.K;
        C.J = R.J;
        C.R = R.op.sh32.R;
        C.QS = C.R >= 64 ? 1 : 2;
        C.defect = defect;
        C.react = x->prob.reaction != 0.0;
        C.force = x->prob.forcing != 0.0;
        const double dt = R.dT / R.J;
        C.dt_react = (float)(dt * x->prob.reaction);
        C.dt_f = (float)(dt * x->prob.forcing);
        C.dTreact = R.dT * x->prob.reaction;
        C.alpha = R.alpha;
        C.tol = tol;
        C.kmax = kmax;
        C.U = R.U;
        C.Udf = R.Udf;
        C.fout = R.fout;
        C.c32 = R.c32;
        C.rs = R.r;
        C.Facc0 = R.Facc2[0];
        C.Facc1 = R.Facc2[1];
        C.p64 = R.p64;
        C.p32 = R.p32;
        C.tab32 = reinterpret_cast<const char*>(R.op.tab32);
        C.u0 = x->u0;
        C.wT = R.op.wT;
        C.dinv64 = R.op.dinv64;
        C.lu64 = R.op.lu64;
        C.dinv32 = R.op.dinv32;
        C.lu32 = R.op.lu32;
        C.wT32 = R.op.wT32;
        C.sc64 = R.sc64;
        C.isc64 = R.isc64;
        C.sc32 = R.sc32;
        C.isc32 = R.isc32;
        C.active = R.active;
        C.iters = R.iters;
        C.status = R.status;
        C.delta = R.delta;
        if (R.op.sh32.W != 0 || R.op.sh32.L != 0 || R.op.sh32.P != 0 || !C.R) return fail(KLECGC_E_CUDA, "batch: a class without the shared-memory fine kernel");
    }
    // task lists, longest first within each stage
    struct Group {
        int R, rt;
        std::vector<BatchTask> t;
    };
    std::vector<Group> fine;
    std::vector<std::pair<double, int>> order(nc);
    for (int c = 0; c < nc; ++c) order[c] = {-(double)hc[c].nx * hc[c].J * hc[c].N, c};
    std::sort(order.begin(), order.end());
    for (auto& oc : order) {
        const BatchClass& C = hc[oc.second];
        const int rt = (C.react || C.force) ? 1 : 0;
        Group* g = nullptr;
        for (auto& x : fine)
            if (x.R == C.R && x.rt == rt) g = &x;
        if (!g) {
            fine.push_back({C.R, rt, {}});
            g = &fine.back();
        }
        const int parts = batch_fine_parts(C.N, C.R);
        for (int64_t s2 = 0; s2 < C.S; ++s2)
            for (int p = 0; p < parts; ++p) g->t.push_back({oc.second, p, s2});
    }
    const int tile = batch_transform_tile(defect);
    std::vector<BatchTask> fwd, inv, solve, inst;
    for (auto& oc : order) {
        const BatchClass& C = hc[oc.second];
        const int tf = (C.nx + tile - 1) / tile, ti = (C.nx + 31) / 32;
        for (int64_t s2 = 0; s2 < C.S; ++s2) {
            for (int p = 0; p < tf; ++p) fwd.push_back({oc.second, p, s2});
            for (int p = 0; p < ti; ++p) inv.push_back({oc.second, p, s2});
            inst.push_back({oc.second, 0, s2});
        }
    }
    {
        std::vector<std::pair<double, int>> byn(nc);
        for (int c = 0; c < nc; ++c) byn[c] = {-(double)hc[c].nx, c};
        std::sort(byn.begin(), byn.end());
        for (auto& oc : byn) {
            const BatchClass& C = hc[oc.second];
            for (int64_t q = 0; q < C.S * C.K; q += 128) solve.push_back({oc.second, (int)q, 0});
        }
    }
    size_t total = fwd.size() + inv.size() + solve.size() + inst.size();
    for (auto& g : fine) total += g.t.size();
    WS(BatchClass, dcls, "batch_cls", nc);
    WS(BatchTask, dtask, "batch_tasks", total);
    const int nq = 3 + (int)fine.size();
    WS(int, queues, "batch_queues", nq);
    WS(int, kdev, "batch_k", 1);
    WS(int, nact, "batch_active", 1);
    TRY(cudaMemcpyAsync(dcls, hc.data(), nc * sizeof(BatchClass), cudaMemcpyHostToDevice, st));
    std::vector<BatchTask> all;
    all.reserve(total);
    std::vector<const BatchTask*> fine_ptr;
    std::vector<int64_t> fine_off;
    for (auto& g : fine) {
        fine_off.push_back((int64_t)all.size());
        all.insert(all.end(), g.t.begin(), g.t.end());
    }
    const int64_t o_fwd = all.size();
    all.insert(all.end(), fwd.begin(), fwd.end());
    const int64_t o_solve = all.size();
    all.insert(all.end(), solve.begin(), solve.end());
    const int64_t o_inv = all.size();
    all.insert(all.end(), inv.begin(), inv.end());
    const int64_t o_inst = all.size();
    all.insert(all.end(), inst.begin(), inst.end());
    TRY(cudaMemcpyAsync(dtask, all.data(), all.size() * sizeof(BatchTask), cudaMemcpyHostToDevice, st));
    const int g_fwd = batch_grid(0, defect), g_solve = batch_grid(1, defect),
              g_inv = batch_grid(2, defect);
    auto iteration = [&](cudaStream_t s2, int k, const int* kd) -> klecgc_status {
        TRY(cudaMemsetAsync(queues, 0, nq * sizeof(int), s2));
        for (size_t g = 0; g < fine.size(); ++g)
            ctx->launch(KLECGC_K_FINE, s2, [&] {
                launch_batch_fine(dcls, dtask + fine_off[g], (int)fine[g].t.size(), queues + 3 + g,
                                  k, kd, fine[g].R, fine[g].rt, 0, s2);
            });
        ctx->launch(KLECGC_K_CGC_FWD, s2, [&] { launch_batch_fwd(defect, dcls, dtask + o_fwd, (int)fwd.size(), queues, k, kd, g_fwd, s2); });
        ctx->launch(KLECGC_K_CGC_SOLVE, s2, [&] { launch_batch_solve(defect, dcls, dtask + o_solve, (int)solve.size(), queues + 1, g_solve, s2); });
        ctx->launch(KLECGC_K_CGC_INV, s2, [&] { launch_batch_inv(defect, dcls, dtask + o_inv, (int)inv.size(), queues + 2, g_inv, s2); });
        TRY(cudaMemsetAsync(nact, 0, sizeof(int), s2));
        ctx->launch(KLECGC_K_CONV, s2, [&] { launch_batch_conv(dcls, dtask + o_inst, (int64_t)inst.size(), k, kd, nact, s2); });
        TRY(cudaGetLastError());
        return KLECGC_OK;
    };
    klecgc_status s = iterate_loop(ctx, st, kdev, nact, 0, kmax, iteration);
    if (s != KLECGC_OK) return s;
    // the classes' results are read on their pool streams
    {
        cudaEvent_t ev;
        TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        TRY(cudaEventRecord(ev, st));
        for (cudaStream_t x : pool) cudaStreamWaitEvent(x, ev, 0);
        cudaEventDestroy(ev);
    }
    (void)n;
    return KLECGC_OK;
}

klecgc_status status_summary(const std::vector<int32_t>& hs, bool capped) {
    bool any_nf = false, any_nc = false;
    for (int32_t v : hs) {
        any_nf |= v == KLECGC_E_NONFINITE;
        any_nc |= v == KLECGC_E_NOT_CONVERGED;
    }
    if (any_nf) return fail(KLECGC_E_NONFINITE, "a sample produced a non-finite iterate");
    if (any_nc)
        return fail(KLECGC_E_NOT_CONVERGED, capped ? "a Krylov solve reached its iteration cap"
                                                   : "a sample did not reach tol within kmax");
    return KLECGC_OK;
}


// Algorithm 2 with the nonlinear CGC (reaction_kind 1 or 2, FP64): per
// iteration, F by Newton steps and the jump b (k_fine_newton), then
// cgc_newton simplified Newton steps of eq. Newton2 from u_0 = U^k, each the
// three diagonalized steps with the averaged Jacobian (k_nl_prep and shifted
// factors with the diagonal extra, or k_nl_prep_burgers and the factors of
// the face couplings; forward transform, solves, inverse transform); the
// last one writes U^{k+1} and the increment norm.
klecgc_status solve_nonlinear(klecgc_ctx* ctx, const double* xi_d, int64_t S, double dT, int J,
                              int N, double alpha, double tol, int kmax, int guess,
                              const double* U_guess, double* U_out, std::vector<int32_t>& hs,
                              std::vector<int32_t>& hi, bool* capped, cudaStream_t st) {
    klecgc_status s;
    const int nx = ctx->nx, K = N / 2 + 1;
    const int64_t NS = S * (int64_t)nx * N;
    const int L = ctx->prob.cgc_newton > 0 ? ctx->prob.cgc_newton : 1;
    const double c = ctx->prob.reaction, f0 = ctx->prob.forcing;
    const int kind = ctx->prob.reaction_kind;
    double *a = nullptr, *wf = nullptr;
    if ((s = nl_weights(ctx, xi_d, S, st, &a, &wf)) != KLECGC_OK) return s;
    WS(double, wT, "wT", S * (int64_t)ctx->nf);
    WS(double, up, "nl_up", S * (int64_t)ctx->nf);
    ctx->launch(KLECGC_K_FIELD, st, [&] { launch_face_weights(a, S, ctx->nf, dT / (ctx->h * ctx->h), wT, st); });
    WS(double, U, "U", NS);
    if (guess == KLECGC_GUESS_GPC) {
        if ((s = gpc_guess_internal(ctx, xi_d, S, true, U, st)) != KLECGC_OK) return s;
    } else if (guess == KLECGC_GUESS_ZERO) {
        TRY(cudaMemsetAsync(U, 0, NS * sizeof(double), st));
    } else if (guess == KLECGC_GUESS_COARSE) {
        bool cap = false;
        if ((s = nl_sequential(ctx, wf, S, N, 1, dT, U, st, &cap)) != KLECGC_OK) return s;
    } else if ((s = import_batch(ctx, U_guess, S, N, U, st)) != KLECGC_OK) {
        return s;
    }
    std::vector<double2> lam;
    double2* lam_d = nullptr;
    if ((s = upload_lambda(ctx, N, alpha, st, lam, &lam_d)) != KLECGC_OK) return s;
    double *sc, *isc;
    if ((s = scale_tables<double>(ctx, N, alpha, st, &sc, &isc)) != KLECGC_OK) return s;
    WS(double, b, "nl_b", NS);
    WS(double, rhs, "r", NS);
    WS(double, ul, "nl_ul", NS);
    WS(double, e, "nl_e", S * (int64_t)nx);
    WS(double, scr, "nl_scratch", 4 * NS);
    WS(Cplx<double>, p64, "p64", S * (int64_t)nx * K);
    WS(Cplx<double>, di, "cgc_dinv64", S * (int64_t)nx * K);
    WS(Cplx<double>, lu, "cgc_lu64", S * (int64_t)nx * K);
    WS(int, active, "active", S);
    WS(int32_t, iters, "iters", S);
    WS(int32_t, status, "status", S);
    WS(unsigned long long, delta, "delta", S);
    WS(int, n_active, "n_active", 1);
    WS(int, ifail, "nl_fail", S);
    WS(unsigned long long, nits, "kry_its", 2);
    TRY(cudaMemsetAsync(nits, 0, 2 * sizeof(unsigned long long), st));
    TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
    TRY(cudaMemsetAsync(iters, 0xff, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(status, 0, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(delta, 0, S * sizeof(unsigned long long), st));
    TRY(cudaMemsetAsync(ifail, 0, S * sizeof(int), st));
    WS(int, kdev, "kdev", 1);
    auto iteration = [&](cudaStream_t st, int k, const int* kd) -> klecgc_status {
        ctx->launch(KLECGC_K_FINE, st, [&] {
            launch_fine_newton(kind, S, N, nx, J, dT, alpha, c, f0, 1, U, ctx->u0, wf, b, scr,
                               active, ifail, nits, st);
        });
        for (int l = 0; l < L; ++l) {
            const double* cur = l == 0 ? U : ul;
            if (kind == 2) {
                // wT receives the lower face couplings lo (k_cgc_solve's wT)
                ctx->launch(KLECGC_K_CGC_FWD, st, [&] { launch_nl_prep_burgers(S, N, nx, dT, c, f0, cur, b, wf, rhs, wT, up, active, st); });
                ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_cgc_factors_faces(S, nx, wT, up, lam_d, K, di, lu, active, st); });
            } else {
                ctx->launch(KLECGC_K_CGC_FWD, st, [&] { launch_nl_prep(S, N, nx, dT, c, f0, cur, b, wf, rhs, e, active, st); });
                ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_cgc_factors<double>(a, S, nx, ctx->h, dT, 0.0, lam_d, K, di, lu, st, e); });
            }
            ctx->launch(KLECGC_K_CGC_FWD, st, [&] { launch_cgc_forward<double, double>(S, N, nx, rhs, sc, p64, active, st); });
            ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] { launch_cgc_solve<double, double>(S, K, nx, di, lu, wT, p64, active, st); });
            if (l + 1 == L)
                ctx->launch(KLECGC_K_CGC_INV, st, [&] { launch_cgc_inverse<double>(S, N, nx, p64, isc, U, 0, delta, nullptr, active, st); });
            else
                ctx->launch(KLECGC_K_CGC_INV, st, [&] { launch_cgc_inverse<double>(S, N, nx, p64, isc, ul, 2, nullptr, nullptr, active, st); });
        }
        TRY(cudaMemsetAsync(n_active, 0, sizeof(int), st));
        ctx->launch(KLECGC_K_CONV, st, [&] { launch_convergence(S, k, kmax, tol, delta, active, iters, status, n_active, st, kd); });
        return KLECGC_OK;
    };
    if ((s = iterate_loop(ctx, st, kdev, n_active, 0, kmax, iteration)) != KLECGC_OK) return s;
    if ((s = export_batch(ctx, U, S, N, U_out, st)) != KLECGC_OK) return s;
    hs.assign(S, 0);
    hi.assign(S, 0);
    std::vector<int> hf(S);
    unsigned long long hn[2] = {0, 0};
    TRY(cudaMemcpyAsync(hs.data(), status, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hi.data(), iters, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hf.data(), ifail, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hn, nits, sizeof(hn), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    ctx->kry_it_fine = hn[0];   // Newton iterations of F and G
    ctx->kry_it_cgc = 0;
    *capped = false;
    for (int64_t i = 0; i < S; ++i)
        if (hf[i] && hs[i] == KLECGC_OK) {
            hs[i] = KLECGC_E_NOT_CONVERGED;
            *capped = true;
        }
    return KLECGC_OK;
}

// Algorithm 1 with Newton propagators (nonlinear problems, FP64): per
// iteration F on every interval (k_fine_newton without the jump), then the
// sequential correction with Newton G (k_parareal_correct_newton).
klecgc_status parareal_nonlinear(klecgc_ctx* ctx, const double* xi_d, int64_t S, double dT,
                                 int J, int N, double tol, int kmax, int guess,
                                 const double* U_guess, double* U_out, std::vector<int32_t>& hs,
                                 std::vector<int32_t>& hi, cudaStream_t st) {
    klecgc_status s;
    const int nx = ctx->nx, kind = ctx->prob.reaction_kind;
    const int64_t NS = S * (int64_t)nx * N;
    const double c = ctx->prob.reaction, f0 = ctx->prob.forcing;
    double *a = nullptr, *wf = nullptr;
    if ((s = nl_weights(ctx, xi_d, S, st, &a, &wf)) != KLECGC_OK) return s;
    WS(double, U, "U", NS);
    if (guess == KLECGC_GUESS_GPC) {
        if ((s = gpc_guess_internal(ctx, xi_d, S, true, U, st)) != KLECGC_OK) return s;
    } else if (guess == KLECGC_GUESS_ZERO) {
        TRY(cudaMemsetAsync(U, 0, NS * sizeof(double), st));
    } else if (guess == KLECGC_GUESS_COARSE) {
        bool cap = false;
        if ((s = nl_sequential(ctx, wf, S, N, 1, dT, U, st, &cap)) != KLECGC_OK) return s;
    } else if ((s = import_batch(ctx, U_guess, S, N, U, st)) != KLECGC_OK) {
        return s;
    }
    WS(double, Fend, "r", NS);
    WS(double, scr, "nl_scratch", 4 * NS);
    WS(double, pscr, "par_scratch_nl", 5 * S * (int64_t)nx);
    WS(int, active, "active", S);
    WS(int32_t, iters, "iters", S);
    WS(int32_t, status, "status", S);
    WS(unsigned long long, delta, "delta", S);
    WS(int, n_active, "n_active", 1);
    WS(int, ifail, "nl_fail", S);
    WS(unsigned long long, nits, "kry_its", 2);
    TRY(cudaMemsetAsync(nits, 0, 2 * sizeof(unsigned long long), st));
    TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
    TRY(cudaMemsetAsync(iters, 0xff, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(status, 0, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(ifail, 0, S * sizeof(int), st));
    WS(int, kdev, "kdev", 1);
    auto iteration = [&](cudaStream_t st, int k, const int* kd) -> klecgc_status {
        ctx->launch(KLECGC_K_FINE, st, [&] {
            launch_fine_newton(kind, S, N, nx, J, dT, 0.0, c, f0, 0, U, ctx->u0, wf, Fend, scr,
                               active, ifail, nits, st);
        });
        ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] {
            launch_parareal_correct_newton(kind, S, N, nx, dT, c, f0, ctx->u0, wf, Fend, U, pscr,
                                           delta, active, ifail, st);
        });
        TRY(cudaMemsetAsync(n_active, 0, sizeof(int), st));
        ctx->launch(KLECGC_K_CONV, st, [&] { launch_convergence(S, k, kmax, tol, delta, active, iters, status, n_active, st, kd); });
        return KLECGC_OK;
    };
    if ((s = iterate_loop(ctx, st, kdev, n_active, 0, kmax, iteration)) != KLECGC_OK) return s;
    if ((s = export_batch(ctx, U, S, N, U_out, st)) != KLECGC_OK) return s;
    hs.assign(S, 0);
    hi.assign(S, 0);
    std::vector<int> hf(S);
    TRY(cudaMemcpyAsync(hs.data(), status, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hi.data(), iters, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hf.data(), ifail, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < S; ++i)
        if (hf[i] && hs[i] == KLECGC_OK) hs[i] = KLECGC_E_NOT_CONVERGED;
    return KLECGC_OK;
}

}  // namespace

extern "C" {

klecgc_status klecgc_solve(klecgc_ctx* ctx, const double* xi, int64_t S, double dT, int32_t J,
                           int32_t N, double alpha, double tol, int32_t kmax, int32_t precision,
                           int32_t guess, const double* U_guess, double* U_out, int32_t* iters_out,
                           int32_t* status_out, void* stream) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    if (S < 0 || (S > 0 && (!xi || !U_out))) return fail(KLECGC_E_INVALID_ARG, "bad array argument");
    if (J < 1 || !(alpha > 0 && alpha < 1) || !(tol > 0) || kmax < 1 || precision < 0 ||
        precision > 2 || guess < 0 || guess > 4 || (guess == KLECGC_GUESS_USER && !U_guess && S > 0))
        return fail(KLECGC_E_INVALID_ARG, "argument out of range");
    if (!pow2_in_range(N)) return fail(KLECGC_E_UNSUPPORTED, "N must be a power of 2 in [2, 64]");
    if ((guess == KLECGC_GUESS_GPC || guess == KLECGC_GUESS_MLP) && N != ctx->N)
        return fail(KLECGC_E_INVALID_ARG, "the gPC and learned guesses need the setup's N");
    if (guess == KLECGC_GUESS_MLP && !ctx->mlp.ready)
        return fail(KLECGC_E_INVALID_ARG, "no network (klecgc_mlp_set / klecgc_mlp_train)");
    if (ctx->dim == 2 && precision == KLECGC_MIXED_DEFECT)
        return fail(KLECGC_E_UNSUPPORTED, "2D: FP64 or MIXED only");
    if (ctx->prob.advection > 0 && precision != KLECGC_FP64)
        return fail(KLECGC_E_UNSUPPORTED, "advection-diffusion: FP64 only");
    if (nonlinear(ctx) && (precision != KLECGC_FP64 || guess == KLECGC_GUESS_MLP))
        return fail(KLECGC_E_UNSUPPORTED, "nonlinear problems: FP64, guesses GPC/ZERO/USER/COARSE");
    klecgc_status s = check_dT(ctx, N, dT);
    if (s != KLECGC_OK) return s;
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;

    const double* xi_d = nullptr;
    if ((s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d)) != KLECGC_OK) return s;
    bool finite = true;
    if ((s = check_xi_finite(ctx, xi_d, S * ctx->M, st, &finite)) != KLECGC_OK) return s;
    if (!finite) {
        if (status_out) {
            std::vector<int32_t> v(S, KLECGC_E_NONFINITE);
            TRY(cudaMemcpyAsync(status_out, v.data(), S * 4, cudaMemcpyDefault, st));
            TRY(cudaStreamSynchronize(st));
        }
        return fail(KLECGC_E_NONFINITE, "xi has a non-finite entry");
    }
    if (nonlinear(ctx)) {
        std::vector<int32_t> hs, hi;
        bool capped = false;
        if ((s = solve_nonlinear(ctx, xi_d, S, dT, J, N, alpha, tol, kmax, guess, U_guess, U_out,
                                 hs, hi, &capped, st)) != KLECGC_OK)
            return s;
        ctx->prof_collect();
        if (iters_out) TRY(cudaMemcpy(iters_out, hi.data(), S * 4, cudaMemcpyDefault));
        if (status_out) TRY(cudaMemcpy(status_out, hs.data(), S * 4, cudaMemcpyDefault));
        return status_summary(hs, capped);
    }
    PinnedInts pin;
    TRY(cudaMallocHost(&pin.p, sizeof(int)));
    SolveRun run;
    run.ctx = ctx;
    run.st = st;
    run.S = S;
    run.N = N;
    run.J = J;
    run.kmax = kmax;
    run.precision = precision;
    run.guess = guess;
    run.dT = dT;
    run.alpha = alpha;
    run.tol = tol;
    run.h_active = pin.p;
    if ((s = run.begin(xi_d, U_guess)) != KLECGC_OK) return s;
    // the first iteration differs (F of the start values, the right-hand side
    // formed rather than accumulated): it runs on its own; iterations k >= 1
    // are one repeated body
    if ((s = run.iterate(st, 0, nullptr)) != KLECGC_OK) return s;
    if ((s = iterate_loop(ctx, st, run.kdev, run.n_active, 1, kmax,
                          [&](cudaStream_t cs, int k, const int* kd) {
                              return run.iterate(cs, k, kd);
                          })) != KLECGC_OK)
        return s;
    std::vector<int32_t> hs, hi;
    bool capped = false;
    if ((s = run.finish(U_out, hs, hi, &capped)) != KLECGC_OK) return s;
    ctx->prof_collect();
    if (iters_out) TRY(cudaMemcpy(iters_out, hi.data(), S * 4, cudaMemcpyDefault));
    if (status_out) TRY(cudaMemcpy(status_out, hs.data(), S * 4, cudaMemcpyDefault));
    return status_summary(hs, capped);
}

klecgc_status klecgc_solve_parareal(klecgc_ctx* ctx, const double* xi, int64_t S, double dT,
                                    int32_t J, int32_t N, double tol, int32_t kmax,
                                    int32_t guess, const double* U_guess, double* U_out,
                                    int32_t* iters_out, int32_t* status_out, void* stream) {
    set_error("");
    if (!ctx) return fail(KLECGC_E_INVALID_ARG, "NULL context");
    if (S < 0 || (S > 0 && (!xi || !U_out))) return fail(KLECGC_E_INVALID_ARG, "bad array argument");
    if (J < 1 || N < 1 || N > 4096 || !(tol > 0) || kmax < 1 || guess < 0 || guess > 3 ||
        (guess == KLECGC_GUESS_USER && !U_guess && S > 0))
        return fail(KLECGC_E_INVALID_ARG, "argument out of range");
    if (ctx->dim != 1) return fail(KLECGC_E_UNSUPPORTED, "classical parareal: 1D problems only");
    if (guess == KLECGC_GUESS_GPC && N != ctx->N)
        return fail(KLECGC_E_INVALID_ARG, "the gPC guess needs the setup's N");
    klecgc_status s = check_dT(ctx, N, dT);
    if (s != KLECGC_OK) return s;
    if (S == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int nx = ctx->nx;
    const int64_t NS = S * (int64_t)nx * N;
    const double* xi_d = nullptr;
    if ((s = stage_in(ctx, xi, (size_t)S * ctx->M, "xi", st, &xi_d)) != KLECGC_OK) return s;
    bool finite = true;
    if ((s = check_xi_finite(ctx, xi_d, S * ctx->M, st, &finite)) != KLECGC_OK) return s;
    if (!finite) return fail(KLECGC_E_NONFINITE, "xi has a non-finite entry");
    if (nonlinear(ctx)) {
        std::vector<int32_t> hs, hi;
        if ((s = parareal_nonlinear(ctx, xi_d, S, dT, J, N, tol, kmax, guess, U_guess, U_out, hs,
                                    hi, st)) != KLECGC_OK)
            return s;
        ctx->prof_collect();
        if (iters_out) TRY(cudaMemcpy(iters_out, hi.data(), S * 4, cudaMemcpyDefault));
        if (status_out) TRY(cudaMemcpy(status_out, hs.data(), S * 4, cudaMemcpyDefault));
        return status_summary(hs, false);
    }
    Operators op;
    if ((s = build_operators(ctx, xi_d, S, N, J, dT, 0.5, 1, 0, st, &op)) != KLECGC_OK) return s;
    WS(FineCoef64, gc, "coarse64", S * (int64_t)(nx + 1));
    ctx->launch(KLECGC_K_FACTORS, st, [&] { launch_fine_factors(op.a, S, nx, ctx->h, dT, ctx->prob.reaction, gc, nullptr, st); });
    WS(double, U, "U", NS);
    if (guess == KLECGC_GUESS_GPC) {
        if ((s = gpc_guess_internal(ctx, xi_d, S, true, U, st)) != KLECGC_OK) return s;
    } else if (guess == KLECGC_GUESS_ZERO) {
        TRY(cudaMemsetAsync(U, 0, NS * sizeof(double), st));
    } else if (guess == KLECGC_GUESS_COARSE) {
        if ((s = coarse_guess_internal(ctx, S, N, dT, op.a, U, st)) != KLECGC_OK) return s;
    } else if ((s = import_batch(ctx, U_guess, S, N, U, st)) != KLECGC_OK) {
        return s;
    }
    WS(double, F, "r", NS);
    WS(double, scr, "par_scratch", 2 * S * (int64_t)nx);
    WS(int, active, "active", S);
    WS(int32_t, iters, "iters", S);
    WS(int32_t, status, "status", S);
    WS(unsigned long long, delta, "delta", S);
    WS(int, n_active, "n_active", 1);
    TRY(cudaMemsetAsync(active, 0xff, S * sizeof(int), st));
    TRY(cudaMemsetAsync(iters, 0xff, S * sizeof(int32_t), st));
    TRY(cudaMemsetAsync(status, 0, S * sizeof(int32_t), st));
    WS(int, kdev, "kdev", 1);
    const double dTf = dT * ctx->prob.forcing;
    auto iteration = [&](cudaStream_t st, int k, const int* kd) -> klecgc_status {
        ctx->launch(KLECGC_K_FINE, st, [&] {
            launch_fine_sweep_fp64(S, N, nx, J, dT, 0.5, ctx->prob.reaction, ctx->prob.forcing, U,
                                   ctx->u0, op.f64, op.wT, F, active, st, 0);
        });
        ctx->launch(KLECGC_K_CGC_SOLVE, st, [&] { launch_parareal_correct(S, N, nx, dTf, ctx->u0, gc, F, U, scr, delta, active, st); });
        TRY(cudaMemsetAsync(n_active, 0, sizeof(int), st));
        ctx->launch(KLECGC_K_CONV, st, [&] { launch_convergence(S, k, kmax, tol, delta, active, iters, status, n_active, st, kd); });
        return KLECGC_OK;
    };
    if ((s = iterate_loop(ctx, st, kdev, n_active, 0, kmax, iteration)) != KLECGC_OK) return s;
    if ((s = export_batch(ctx, U, S, N, U_out, st)) != KLECGC_OK) return s;
    std::vector<int32_t> hs(S), hi(S);
    TRY(cudaMemcpyAsync(hs.data(), status, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaMemcpyAsync(hi.data(), iters, S * 4, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    ctx->prof_collect();
    if (iters_out) TRY(cudaMemcpy(iters_out, hi.data(), S * 4, cudaMemcpyDefault));
    if (status_out) TRY(cudaMemcpy(status_out, hs.data(), S * 4, cudaMemcpyDefault));
    return status_summary(hs, false);
}

klecgc_status klecgc_solve_batch(klecgc_ctx* const* ctxs, int32_t n_ctx,
                                 const klecgc_instance* inst, int64_t n, const double* xi,
                                 double alpha, double tol, int32_t kmax, int32_t precision,
                                 int32_t guess, double* U_out, int32_t* iters_out,
                                 int32_t* status_out, void* stream) {
    set_error("");
    if (!ctxs || n_ctx < 1 || n < 0 || (n > 0 && (!inst || !xi || !U_out)))
        return fail(KLECGC_E_INVALID_ARG, "bad argument");
    if (!(alpha > 0 && alpha < 1) || !(tol > 0) || kmax < 1 || precision < 0 || precision > 2 ||
        !(guess == KLECGC_GUESS_GPC || guess == KLECGC_GUESS_ZERO || guess == KLECGC_GUESS_COARSE))
        return fail(KLECGC_E_INVALID_ARG, "argument out of range (batch guesses: GPC, ZERO, COARSE)");
    int dev = 0;
    TRY(cudaGetDevice(&dev));
    const int M = ctxs[0] ? ctxs[0]->M : 0;
    for (int c = 0; c < n_ctx; ++c) {
        const klecgc_ctx* x = ctxs[c];
        if (!x || !x->basis) return fail(KLECGC_E_INVALID_ARG, "NULL context");
        if (x->device != dev) return fail(KLECGC_E_INVALID_ARG, "every context must be on the current device");
        if (x->M != M) return fail(KLECGC_E_INVALID_ARG, "every context must have the same M");
        if (x->dim == 2 && precision == KLECGC_MIXED_DEFECT)
            return fail(KLECGC_E_UNSUPPORTED, "2D: FP64 or MIXED only");
        if (x->prob.advection > 0 && precision != KLECGC_FP64)
            return fail(KLECGC_E_UNSUPPORTED, "advection-diffusion: FP64 only");
        if (nonlinear(x)) return fail(KLECGC_E_UNSUPPORTED, "the batch takes linear problems");
    }
    for (int64_t i = 0; i < n; ++i)
        if (inst[i].ctx < 0 || inst[i].ctx >= n_ctx || inst[i].J < 1)
            return fail(KLECGC_E_INVALID_ARG, "instance " + std::to_string(i) + ": bad ctx index or J");
    if (n == 0) return KLECGC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    klecgc_ctx* c0 = ctxs[0];
    klecgc_status s;

    // packed output offsets, classes of equal (context, J), largest work first
    std::vector<int64_t> off(n);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        off[i] = total;
        total += (int64_t)ctxs[inst[i].ctx]->N * ctxs[inst[i].ctx]->ns;
    }
    std::map<std::pair<int, int>, std::vector<int64_t>> groups;
    for (int64_t i = 0; i < n; ++i) groups[{inst[i].ctx, inst[i].J}].push_back(i);
    struct Cls {
        int ci, J;
        std::vector<int64_t> ids;
        double work;
    };
    std::vector<Cls> cls;
    for (auto& g : groups) {
        const klecgc_ctx* x = ctxs[g.first.first];
        cls.push_back({g.first.first, g.first.second, g.second,
                       (double)g.second.size() * x->N * x->ns * g.first.second});
    }
    std::stable_sort(cls.begin(), cls.end(), [](const Cls& a, const Cls& b) { return a.work > b.work; });
    const int nc = (int)cls.size();

    const double* xi_d = nullptr;
    if ((s = stage_in(c0, xi, (size_t)n * M, "batch_xi", st, &xi_d)) != KLECGC_OK) return s;
    bool finite = true;
    if ((s = check_xi_finite(c0, xi_d, n * M, st, &finite)) != KLECGC_OK) return s;
    if (!finite) {
        if (status_out) {
            std::vector<int32_t> v(n, KLECGC_E_NONFINITE);
            TRY(cudaMemcpyAsync(status_out, v.data(), n * 4, cudaMemcpyDefault, st));
            TRY(cudaStreamSynchronize(st));
        }
        return fail(KLECGC_E_NONFINITE, "xi has a non-finite entry");
    }

    // a pool of streams ordered after the caller's stream
    struct Pool {
        std::vector<cudaStream_t> s;
        cudaEvent_t ev = nullptr;
        ~Pool() {
            for (cudaStream_t x : s) cudaStreamDestroy(x);
            if (ev) cudaEventDestroy(ev);
        }
    } pool;
    const int P = std::min(nc, 8);
    TRY(cudaEventCreateWithFlags(&pool.ev, cudaEventDisableTiming));
    TRY(cudaEventRecord(pool.ev, st));
    for (int i = 0; i < P; ++i) {
        cudaStream_t x;
        TRY(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        pool.s.push_back(x);
        TRY(cudaStreamWaitEvent(x, pool.ev, 0));
    }
    PinnedInts pin;
    TRY(cudaMallocHost(&pin.p, nc * sizeof(int)));
    // MIXED / MIXED_DEFECT in 1D: all classes advance together, each stage one
    // persistent launch over every class (batch_persistent); otherwise the
    // classes step in lockstep on the stream pool
    bool persistent = precision != KLECGC_FP64;
    for (int c = 0; c < n_ctx; ++c) persistent &= ctxs[c]->dim == 1;
    std::vector<SolveRun> runs(nc);
    for (int c = 0; c < nc; ++c) {
        SolveRun& R = runs[c];
        R.ctx = ctxs[cls[c].ci];
        R.tag = "#b" + std::to_string(c);
        R.st = pool.s[c % P];
        R.S = (int64_t)cls[c].ids.size();
        R.N = R.ctx->N;
        R.J = cls[c].J;
        R.kmax = kmax;
        R.precision = precision;
        R.guess = guess;
        R.dT = R.ctx->prob.T / R.N;
        R.alpha = alpha;
        R.tol = tol;
        R.h_active = pin.p + c;
        klecgc_ctx* ctx = R.ctx;
        double* xic = nullptr;
        {
            TagScope ts(ctx, R.tag);
            WS(double, xg, "bxi", R.S * M);
            WS(int64_t, idx, "bidx", R.S);
            TRY(cudaMemcpyAsync(idx, cls[c].ids.data(), R.S * sizeof(int64_t), cudaMemcpyHostToDevice, R.st));
            launch_gather_rows(xi_d, idx, R.S, M, xg, R.st);
            xic = xg;
        }
        ctx->fine_smem_only = persistent;
        s = R.begin(xic, nullptr);
        ctx->fine_smem_only = false;
        if (s != KLECGC_OK) return s;
    }
    if (persistent) {
        if ((s = batch_persistent(c0, runs, n, kmax, tol, st, pool.s)) != KLECGC_OK) return s;
    } else {
        // iterations in lockstep: every class still active enqueues one step,
        // then the host reads each class's active count
        std::vector<char> done(nc, 0);
        for (int left = nc; left > 0;) {
            for (int c = 0; c < nc; ++c)
                if (!done[c] && (s = runs[c].step()) != KLECGC_OK) return s;
            for (int c = 0; c < nc; ++c) {
                if (done[c]) continue;
                TRY(cudaStreamSynchronize(runs[c].st));
                if (runs[c].finished()) {
                    done[c] = 1;
                    --left;
                }
            }
        }
    }
    // results: class blocks scattered to the packed per-instance layout
    const bool dev_out = is_device_ptr(U_out);
    double* dst = U_out;
    if (!dev_out) {
        klecgc_ctx* ctx = c0;
        WS(double, big, "batch_out", total);
        dst = big;
    }
    std::vector<int32_t> hs_all(n), hi_all(n);
    bool capped_any = false;
    for (int c = 0; c < nc; ++c) {
        SolveRun& R = runs[c];
        klecgc_ctx* ctx = R.ctx;
        const int64_t block = (int64_t)R.N * ctx->ns;
        double* tmp = nullptr;
        int64_t* offd = nullptr;
        {
            TagScope ts(ctx, R.tag);
            WS(double, t, "bU", R.S * block);
            WS(int64_t, o, "boff", R.S);
            tmp = t;
            offd = o;
        }
        std::vector<int32_t> hs, hi;
        bool capped = false;
        if ((s = R.finish(tmp, hs, hi, &capped)) != KLECGC_OK) return s;
        capped_any |= capped;
        std::vector<int64_t> oh(R.S);
        for (int64_t j = 0; j < R.S; ++j) {
            const int64_t i = cls[c].ids[j];
            oh[j] = off[i];
            hs_all[i] = hs[j];
            hi_all[i] = hi[j];
        }
        TRY(cudaMemcpyAsync(offd, oh.data(), R.S * sizeof(int64_t), cudaMemcpyHostToDevice, R.st));
        ctx->launch(KLECGC_K_LAYOUT, R.st, [&] { launch_scatter_blocks(tmp, offd, R.S, block, dst, R.st); });
        TRY(cudaGetLastError());
    }
    for (cudaStream_t x : pool.s) TRY(cudaStreamSynchronize(x));
    if (!dev_out) TRY(cudaMemcpy(U_out, dst, total * sizeof(double), cudaMemcpyDeviceToHost));
    for (int c = 0; c < n_ctx; ++c) ctxs[c]->prof_collect();
    if (iters_out) TRY(cudaMemcpy(iters_out, hi_all.data(), n * 4, cudaMemcpyDefault));
    if (status_out) TRY(cudaMemcpy(status_out, hs_all.data(), n * 4, cudaMemcpyDefault));
    return status_summary(hs_all, capped_any);
}

}  // extern "C"
