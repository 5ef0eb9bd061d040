// Surrogate guess on the fifth-generation tensor cores (Algorithm 3 step 6):
//   U[s][c] = ubar[c] + sum_j psi[s][j] W[j][c].
//
// One CTA computes a 128 x 256 output tile with tcgen05.mma (kind::tf32, FP32
// accumulation in tensor memory).  To keep FP32 accuracy each operand is
// split into a TF32 head and an FP32 tail, x = hi + lo (k_split_tf32), and the
// tile accumulates hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32
// rounding).  K-chunks of 32 of the four operands (psi head / tail 128 x 32,
// W^T head / tail 256 x 32) arrive by TMA (cp.async.bulk.tensor, 128-byte
// swizzle) into a two-stage shared-memory ring; one thread issues the loads,
// one thread issues the MMAs and commits them to the stage's "empty"
// mbarrier.  Every wait on an mbarrier is bounded by a clock budget, after
// which the CTA sets the error flag, drains its copies and MMAs in flight
// (again bounded) and frees its tensor memory before it returns.  The
// epilogue adds ubar in FP64, or, for the mixed-defect path, adds the FP32
// accumulator to a pair copy of ubar in double-float arithmetic and stores
// U directly as FP32 pairs (hi, lo).
//
// Shared-memory layout of one operand chunk (R rows of 32 FP32 = 128 bytes):
// row r at byte 128 r with its eight 16-byte pieces permuted by the 128-byte
// swizzle (piece q of row r stored at piece q ^ (r % 8)); the 8-row groups are
// 1024 bytes apart, the stride byte offset of the matrix descriptor.
#include <cuda.h>  // CUtensorMap and the encode function's type (resolved at run time)

#include <cstdint>
#include <mutex>

#include <cuda_bf16.h>

#include "common.cuh"

namespace klecgc {

namespace {

constexpr int TM = 128, TN = 256, TK = 32;
constexpr int A_BYTES = TM * TK * 4, B_BYTES = TN * TK * 4;   // one split half
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;          // hi and lo of A and B
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 64 + 1024;   // + alignment of the stages
constexpr long long kWaitCycles = 200000000LL;                   // ~0.1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false when the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Loads 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory descriptor of a K-major operand tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes (32 FP32), 8-row groups 1024 bytes apart
// (stride byte offset), layout type 2 (SWIZZLE_128B), descriptor version 1;
// the leading byte offset is unused for this layout (set to 16 bytes).  The
// K step inside the 128-byte row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 2D tiled TMA load of box (x, y) into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// One CTA per 128 x 256 output tile.  Warp 0 (one thread) loads the four
// operand tiles of each K-chunk (psi head / tail 128 x 32, W^T head / tail
// 256 x 32) by TMA into a stage and arms its "full" barrier with the byte
// count; warp 1 (one thread) waits on "full", issues the twelve MMAs of the
// chunk and commits them to the stage's "empty" barrier, which the producer
// waits on before it refills the stage.  All waits are bounded.
__global__ void __launch_bounds__(128, 1) k_guess_tc(int64_t S, int64_t NC, int Kp,
                                                    const __grid_constant__ CUtensorMap mAh,
                                                    const __grid_constant__ CUtensorMap mAl,
                                                    const __grid_constant__ CUtensorMap mBh,
                                                    const __grid_constant__ CUtensorMap mBl,
                                                    const double* __restrict__ ubar,
                                                    const float2* __restrict__ ubar_df,
                                                    double* __restrict__ U,
                                                    int* __restrict__ err) {
    extern __shared__ __align__(1024) char smem_raw[];
    // 1024-byte alignment of the stages (the swizzle atoms)
    char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);   // [2]
    uint64_t* empty = full + 2;                                              // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + 2);
    int* flags = reinterpret_cast<int*>(tslot + 1);   // [0] skip, [1] loads issued, [2] chunks committed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // row tiles vary fastest: the CTAs that share a W^T tile run together and
    // read it from L2 (W^T is larger than L2 at the bench sizes)
    const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TN;
    // once a CTA has timed out the launch's result is void: later CTAs skip
    // (read by one thread so that the whole CTA takes the same branch)
    if (threadIdx.x == 0) flags[0] = *reinterpret_cast<volatile int*>(err);
    __syncthreads();
    if (flags[0]) return;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = make_idesc(TM, TN);
    const int nch = Kp / TK;
    bool ok = true;

    int issued = 0, committed = 0;
    if (warp == 0 && lane == 0) {
        // producer
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c & 1;
            char* base = smem + st * STAGE_BYTES;
            if (c >= 2) ok = mbar_wait(&empty[st], ((c - 2) >> 1) & 1);
            if (!ok) break;
            mbar_expect_tx(&full[st], STAGE_BYTES);
            tma_load_2d(base, &mAh, c * TK, (int)m0, &full[st]);
            tma_load_2d(base + A_BYTES, &mAl, c * TK, (int)m0, &full[st]);
            tma_load_2d(base + 2 * A_BYTES, &mBh, c * TK, (int)n0, &full[st]);
            tma_load_2d(base + 2 * A_BYTES + B_BYTES, &mBl, c * TK, (int)n0, &full[st]);
            issued = c + 1;
        }
        flags[1] = issued;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c & 1;
            char* base = smem + st * STAGE_BYTES;
            ok = mbar_wait(&full[st], (c >> 1) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah0 = smem_u32(base), al0 = smem_u32(base + A_BYTES);
            const uint32_t bh0 = smem_u32(base + 2 * A_BYTES);
            const uint32_t bl0 = smem_u32(base + 2 * A_BYTES + B_BYTES);
#pragma unroll
            for (int kk = 0; kk < TK / 8; ++kk) {
                const uint32_t ko = kk * 32;   // 8 TF32 values per K step
                const uint64_t ah = make_desc_sw128(ah0 + ko), al = make_desc_sw128(al0 + ko);
                const uint64_t bh = make_desc_sw128(bh0 + ko), bl = make_desc_sw128(bl0 + ko);
                mma_tf32(tmem, ah, bh, idesc, (c | kk) ? 1u : 0u);
                mma_tf32(tmem, ah, bl, idesc, 1u);
                mma_tf32(tmem, al, bh, idesc, 1u);
            }
            mma_commit(&empty[st]);
            committed = c + 1;
        }
        flags[2] = committed;
    }
    ok = __syncthreads_and(ok);
    issued = flags[1];
    committed = flags[2];
    // every thread: the last commit of each stage has landed (all MMAs done);
    // on failure also every TMA load still in flight, so that nothing writes
    // shared memory or tensor memory after the CTA has left
    bool done = true;
    for (int c = committed - 2; c < committed; ++c)
        if (c >= 0) done = mbar_wait(&empty[c & 1], (c >> 1) & 1) && done;
    if (!ok)
        for (int c = issued - 2; c < issued; ++c)
            if (c >= committed && c >= 0) done = mbar_wait(&full[c & 1], (c >> 1) & 1) && done;
    ok = __syncthreads_and(ok && done && committed == nch);   // uniform: TMEM loads are warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok) {
        // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
        const int64_t row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < TN; cb += 32) {
            float v[32];
            tmem_ld32(lane_addr + cb, v);
            if (row < S) {
                double* out = U + row * NC + n0 + cb;
                if (ubar_df && n0 + cb + 32 <= NC) {
                    // U as FP32 pairs: ubar's pair plus the FP32 accumulator,
                    // added in double-float arithmetic (FP32 pipes only)
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const float4 b = *reinterpret_cast<const float4*>(ubar_df + n0 + cb + i);
                        const float2 p0 = df_add(make_float2(b.x, b.y), v[i]);
                        const float2 p1 = df_add(make_float2(b.z, b.w), v[i + 1]);
                        *reinterpret_cast<float4*>(out + i) = make_float4(p0.x, p0.y, p1.x, p1.y);
                    }
                } else if (ubar_df) {
                    float2* outp = reinterpret_cast<float2*>(out);
                    for (int i = 0; i < 32 && n0 + cb + i < NC; ++i)
                        outp[i] = df_add(ubar_df[n0 + cb + i], v[i]);
                } else if (n0 + cb + 32 <= NC) {
#pragma unroll
                    for (int i = 0; i < 32; i += 2) {
                        const double2 b = *reinterpret_cast<const double2*>(ubar + n0 + cb + i);
                        *reinterpret_cast<double2*>(out + i) =
                            make_double2(b.x + (double)v[i], b.y + (double)v[i + 1]);
                    }
                } else {
                    for (int i = 0; i < 32 && n0 + cb + i < NC; ++i)
                        out[i] = ubar[n0 + cb + i] + (double)v[i];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                     : "memory");
}

// hi = TF32 rounding of x, lo = x - hi (exact), elementwise.
// Elementwise, so x may alias hi (in-place split).
__global__ void k_split_tf32(const float* x, int64_t n, float* hi, float* __restrict__ lo) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float v = x[t], h = tf32_hi(v);
    hi[t] = h;
    lo[t] = v - h;
}

// out[c][j] = in[j][c] for j < P, 0 for P <= j < Kp (W^T, K-major for the MMA).
__global__ void k_pad_transpose(const float* __restrict__ in, int P, int64_t NC, int Kp,
                                float* __restrict__ out) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = j0 + y;
        const int64_t c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (j < P && c < NC) ? in[(int64_t)j * NC + c] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int64_t c = c0 + y;
        const int j = j0 + threadIdx.x;
        if (c < NC && j < Kp) out[c * Kp + j] = tile[threadIdx.x][y];
    }
}

}  // namespace

int guess_tc_k_padded(int P) { return (P + TK - 1) / TK * TK; }

void launch_pad_transpose(const float* W, int P, int64_t NC, int Kp, float* Wt, cudaStream_t st) {
    if (NC == 0) return;
    dim3 grid((unsigned)((NC + 31) / 32), (unsigned)((Kp + 31) / 32));
    k_pad_transpose<<<grid, dim3(32, 8), 0, st>>>(W, P, NC, Kp, Wt);
}

void launch_split_tf32(const float* x, int64_t n, float* hi, float* lo, cudaStream_t st) {
    if (n == 0) return;
    k_split_tf32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, hi, lo);
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// [rows][Kp] FP32, box 32 x box_rows, 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* m, const float* base, int64_t rows, int Kp, int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
    const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace

// ---- BF16 GEMM on the tensor cores for the learned guess's network
// C[m][n] = sum_k A[m][k] B[n][k] (both operands BF16, K-major), FP32
// accumulation in tensor memory (tcgen05.mma kind::f16 with BF16 A and B),
// one 128 x 128 output tile per CTA, K-chunks of 64 (one 128-byte swizzle
// row) by TMA into a four-stage ring: the same producer / MMA-issuer /
// bounded-wait structure as k_guess_tc.  Epilogue: v = acc (+ bias[n]);
// zmask: v = 0 where zmask[m][n] <= 0 (the ReLU derivative); C (FP32) and/or
// Cb (BF16, ReLU applied when relu).
namespace {

constexpr int GM = 128, GN = 128, GK = 64, GSTAGES = 4;
constexpr int GA_BYTES = GM * GK * 2, GB_BYTES = GN * GK * 2;
constexpr int GSTAGE_BYTES = GA_BYTES + GB_BYTES;
constexpr int GSMEM_BYTES = GSTAGES * GSTAGE_BYTES + 128 + 1024;

// Instruction descriptor of kind::f16: D FP32 (bit 4), A and B BF16 (format
// 1 at bits 7 and 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__global__ void __launch_bounds__(128, 1) k_gemm_bf16_tc(int M, int N, int K,
                                                        const __grid_constant__ CUtensorMap mA,
                                                        const __grid_constant__ CUtensorMap mB,
                                                        const float* __restrict__ bias,
                                                        const float* __restrict__ zmask, int ldz,
                                                        float* __restrict__ C, int ldc,
                                                        __nv_bfloat16* __restrict__ Cb, int ldcb,
                                                        int relu, int* __restrict__ err) {
    extern __shared__ __align__(1024) char smem_raw[];
    char* smem = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + GSTAGES * GSTAGE_BYTES);   // [GSTAGES]
    uint64_t* empty = full + GSTAGES;                                              // [GSTAGES]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(empty + GSTAGES);
    int* flags = reinterpret_cast<int*>(tslot + 1);   // [0] skip, [1] issued, [2] committed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    if (threadIdx.x == 0) flags[0] = *reinterpret_cast<volatile int*>(err);
    __syncthreads();
    if (flags[0]) return;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(GN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < GSTAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = make_idesc_bf16(GM, GN);
    const int nch = (K + GK - 1) / GK;
    bool ok = true;
    int issued = 0, committed = 0;
    if (warp == 0 && lane == 0) {
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c % GSTAGES;
            char* base = smem + st * GSTAGE_BYTES;
            if (c >= GSTAGES) ok = mbar_wait(&empty[st], ((c - GSTAGES) / GSTAGES) & 1);
            if (!ok) break;
            mbar_expect_tx(&full[st], GSTAGE_BYTES);
            tma_load_2d(base, &mA, c * GK, m0, &full[st]);
            tma_load_2d(base + GA_BYTES, &mB, c * GK, n0, &full[st]);
            issued = c + 1;
        }
        flags[1] = issued;
    } else if (warp == 1 && lane == 0) {
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c % GSTAGES;
            char* base = smem + st * GSTAGE_BYTES;
            ok = mbar_wait(&full[st], (c / GSTAGES) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(base), b0 = smem_u32(base + GA_BYTES);
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk) {
                const uint32_t ko = kk * 32;   // 16 BF16 values per K step
                mma_bf16(tmem, make_desc_sw128(a0 + ko), make_desc_sw128(b0 + ko), idesc,
                         (c | kk) ? 1u : 0u);
            }
            mma_commit(&empty[st]);
            committed = c + 1;
        }
        flags[2] = committed;
    }
    ok = __syncthreads_and(ok);
    issued = flags[1];
    committed = flags[2];
    bool done = true;
    for (int c = committed - GSTAGES; c < committed; ++c)
        if (c >= 0) done = mbar_wait(&empty[c % GSTAGES], (c / GSTAGES) & 1) && done;
    if (!ok)
        for (int c = issued - GSTAGES; c < issued; ++c)
            if (c >= committed && c >= 0) done = mbar_wait(&full[c % GSTAGES], (c / GSTAGES) & 1) && done;
    ok = __syncthreads_and(ok && done && committed == nch);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int cb = 0; cb < GN; cb += 32) {
            float v[32];
            tmem_ld32(lane_addr + cb, v);
            if (row < M) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int n = n0 + cb + i;
                    if (n >= N) break;
                    float x = v[i];
                    if (bias) x += bias[n];
                    if (zmask && !(zmask[(int64_t)row * ldz + n] > 0.f)) x = 0.f;
                    if (C) C[(int64_t)row * ldc + n] = x;
                    if (Cb) Cb[(int64_t)row * ldcb + n] = __float2bfloat16(relu ? fmaxf(x, 0.f) : x);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GN)
                     : "memory");
}

// out[c][r] = in[r][c] for an R x Cc BF16 matrix (leading dimension ld_in).
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ in, int R, int Cc, int ld_in,
                                 __nv_bfloat16* __restrict__ out) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < R && c < Cc) ? in[(int64_t)r * ld_in + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (c < Cc && r < R) out[(int64_t)c * R + r] = tile[threadIdx.x][y];
    }
}

// [rows][K] BF16 (row stride ld elements), box 64 x box_rows, 128-byte swizzle.
bool make_map_bf16(CUtensorMap* m, const __nv_bfloat16* base, int64_t rows, int K, int ld,
                   int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)GK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace

void launch_transpose_bf16(const __nv_bfloat16* in, int R, int Cc, int ld_in, __nv_bfloat16* out,
                           cudaStream_t st) {
    if (R == 0 || Cc == 0) return;
    dim3 grid((unsigned)((Cc + 31) / 32), (unsigned)((R + 31) / 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(in, R, Cc, ld_in, out);
}

bool gemm_bf16_tc_ok(int M, int N, int K, const void* A, int lda, const void* B, int ldb) {
    // TMA: 16-byte aligned bases, row strides a multiple of 16 bytes; at least
    // one full K-chunk and one tile in M
    return M >= 64 && N >= 32 && K >= GK && (lda % 8) == 0 && (ldb % 8) == 0 &&
           (reinterpret_cast<uintptr_t>(A) % 16) == 0 && (reinterpret_cast<uintptr_t>(B) % 16) == 0;
}

cudaError_t launch_gemm_bf16_tc(int M, int N, int K, const __nv_bfloat16* A, int lda,
                                const __nv_bfloat16* B, int ldb, const float* bias,
                                const float* zmask, int ldz, float* C, int ldc,
                                __nv_bfloat16* Cb, int ldcb, bool relu, int* err,
                                cudaStream_t st) {
    if (M == 0 || N == 0) return cudaSuccess;
    CUtensorMap mA, mB;
    if (!make_map_bf16(&mA, A, M, K, lda, GM) || !make_map_bf16(&mB, B, N, K, ldb, GN))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GSMEM_BYTES);
        attr = true;
    }
    dim3 grid((unsigned)((M + GM - 1) / GM), (unsigned)((N + GN - 1) / GN));
    k_gemm_bf16_tc<<<grid, 128, GSMEM_BYTES, st>>>(M, N, K, mA, mB, bias, zmask, ldz, C, ldc, Cb,
                                                   ldcb, relu ? 1 : 0, err);
    return cudaGetLastError();
}

cudaError_t launch_guess_tc(int64_t S, int64_t NC, int Kp, const float* psi_hi,
                            const float* psi_lo, const float* Wt_hi, const float* Wt_lo,
                            const double* ubar, const float2* ubar_df, double* U, int* err,
                            cudaStream_t st) {
    if (S == 0 || NC == 0) return cudaSuccess;
    CUtensorMap mAh, mAl, mBh, mBl;
    if (!make_map(&mAh, psi_hi, S, Kp, TM) || !make_map(&mAl, psi_lo, S, Kp, TM) ||
        !make_map(&mBh, Wt_hi, NC, Kp, TN) || !make_map(&mBl, Wt_lo, NC, Kp, TN))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_guess_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        attr = true;
    }
    const int64_t tiles_n = (NC + TN - 1) / TN;
    if (tiles_n > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((S + TM - 1) / TM), (unsigned)tiles_n);
    k_guess_tc<<<grid, 128, SMEM_BYTES, st>>>(S, NC, Kp, mAh, mAl, mBh, mBl, ubar, ubar_df, U, err);
    return cudaGetLastError();
}

}  // namespace klecgc
