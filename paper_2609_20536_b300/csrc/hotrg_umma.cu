// Split-precision contraction engine on the 5th-generation tensor cores
// (tcgen05, sm_103a): C = A B^T for FP64 (or FP32-pair) operands, computed
// from fixed-point BF16 slices whose products accumulate exactly.
//
// Slicing (per row of A and per row of B, i.e. per output row / column):
//   e      = exponent with max_k |X_k| < 2^e (a power of two per row)
//   F_k    = round(X_k 2^(T - e)), a signed integer, T = 7 + 8 (NS - 1) bits
//   digits = NS balanced digits c_0 .. c_{NS-1}, |c_p| <= 128, F = sum c_p 2^(8(NS-1-p))
//   slice p holds c_p 2^(-8p): at most 8 significant bits, exact in BF16.
// The tensor cores accumulate in FP32 by truncation, so only sums that stay
// exactly representable are safe.  Every slice product is an integer (times a
// power of two) of magnitude <= 2^14.  Over a chunk of 512 values of k the
// diagonal-0 sum (c_0 c_0', one product per k) and the diagonal-1 sum
// (c_0 c_1' + c_1 c_0') stay <= 2^24 and are exact; diagonals p + q >= 2 sit
// 2^-16 below the leading term and go to a third accumulator whose FP32
// error is below 2^-28 of the result.  After each chunk the epilogue warps
// fold the three TMEM accumulators into per-element double-float running
// sums (error-free TwoSum), then hand TMEM back for the next chunk.  Pairs
// with p + q > NS - 1 are dropped (2^-8NS below the leading term).  Result:
//   C = (hi + lo) 2^(eA + eB - 14).
//
// The GEMM kernel: one CTA per 128 x 128 output tile.  Warp 0 issues TMA loads
// (all NS slices of a 128 x 32 A tile and a 128 x 32 B tile per stage, 64-byte
// swizzle), warp 1 issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32 in TMEM),
// warps 2..9 drain the accumulators per chunk.  Every mbarrier wait is
// bounded; on timeout the kernel records HOTRG_ETIMEOUT in a device status
// word, other CTAs see it and leave, and each CTA drains its own copies first.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace hotrg {

// ---------------------------------------------------------------------------
// output / input element formats of the engine
// ---------------------------------------------------------------------------
enum ElemFmt : int { FMT_F64 = 0, FMT_F32PAIR = 1 };

// Bits of the leading digit and the K extent of one exactly-accumulated chunk:
// with |c| <= 128 every slice product is at most 2^14, so the diagonal-0 sum
// (one product per k) and the diagonal-1 sum (two products per k) over 512
// values of k stay within 2^24 and are exact in FP32.
constexpr int SLICE_B1 = 7;
constexpr int KCHUNK = 512;

// ---------------------------------------------------------------------------
// Slicing kernel: one warp per row.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int exp_f64(double v) {  // floor(log2 |v|) for normal v; -2000 for 0
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return -2000;  // zero or subnormal: treated as zero
    return ex - 1023;
}

__device__ __forceinline__ int exp_f32(float v) {
    const uint32_t b = __float_as_uint(v);
    const int ex = (int)((b >> 23) & 0xff);
    if (ex == 0) return -2000;
    return ex - 127;
}

// round(|v| 2^sh) as an unsigned 64-bit integer, for |v| 2^sh < 2^62 (FP64 input)
__device__ __forceinline__ uint64_t fixed_f64(double v, int sh) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;
    const uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const int s = ex - 1075 + sh;  // value = mant 2^(ex - 1075), times 2^sh
    if (s >= 0) return s >= 10 ? 0 : (mant << s);  // not reached for |v| 2^sh < 2^62
    const int r = -s;
    if (r >= 63) return 0;
    return (mant + (1ull << (r - 1))) >> r;
}

// round(|v| 2^sh) with v's sign, from an FP32 bit pattern (|v| 2^sh < 2^39; 0 for zero or
// subnormal v).
__device__ __forceinline__ int64_t fixed_half(uint32_t b, int sh) {
    const int ex = (int)((b >> 23) & 0xff);
    if (ex == 0) return 0;
    const uint32_t mant = (b & 0x7fffffu) | 0x800000u;
    const int s = ex - 150 + sh;
    int64_t a;
    if (s >= 0) {
        a = s >= 39 ? 0 : ((int64_t)mant << s);
    } else {
        const int r = -s;
        a = r > 24 ? 0 : (int64_t)((mant + (1u << (r - 1))) >> r);  // below 1/2 when r > 24
    }
    return (b >> 31) ? -a : a;
}

// Fixed-point value F = round(v 2^sh) of one element from its 8-byte pattern: an FP64 value,
// or an exact FP32 pair hi + lo (hi in the low word, |lo| <= ulp(hi) / 2).  For a pair the two
// parts are rounded on their own: |hi| 2^sh is an integer whenever |hi| >= 2^(23 - sh), which
// with five slices (sh = 39 - e for a row whose largest element lies below 2^e) covers every
// element within 2^-15 of the largest, so F is then exact; for the smaller ones the second
// rounding adds at most half a unit, the size of the largest element's own rounding error.
template <int FMT>
__device__ __forceinline__ int64_t fixed_elem(uint64_t bits, int sh) {
    if (FMT == FMT_F64) {
        const int64_t a = (int64_t)fixed_f64(__longlong_as_double((long long)bits), sh);
        return (bits >> 63) ? -a : a;  // the sign from the bit pattern (no FP64 compare)
    } else {
        return fixed_half((uint32_t)(bits & 0xffffffffu), sh) + fixed_half((uint32_t)(bits >> 32), sh);
    }
}

// The NS balanced base-256 digits of F (|F| <= 2^(B1 + 8 (NS - 1))): c_0 = round(F / 2^(8 (NS - 1))),
// each later digit the rounded remainder (round half up), the last the exact remainder, so
// |c_p| <= 128.  After c_0 the remainder fits 32 bits.  bits[p] = the BF16 pattern of
// c_p 2^(-8p): c_p has at most 8 significant bits, so its FP32 value truncates to BF16 exactly.
__device__ __forceinline__ void slice_digits(int64_t F, int NS, uint32_t* bits) {
    const int sh0 = 8 * (NS - 1);
    const int64_t c0 = (F >> sh0) + ((F >> (sh0 - 1)) & 1);
    int32_t r = (int32_t)(F - (c0 << sh0));
    bits[0] = __float_as_uint((float)c0) >> 16;
    float scale = 1.0f;
#pragma unroll
    for (int p = 1; p < 5; ++p) {
        if (p < NS) {
            const int sh = 8 * (NS - 1 - p);
            int32_t c;
            if (sh == 0) {
                c = r;
            } else {
                c = (r >> sh) + ((r >> (sh - 1)) & 1);
                r = (int32_t)((uint32_t)r - ((uint32_t)c << sh));  // exact: the result fits
            }
            scale *= 1.0f / 256.0f;
            bits[p] = __float_as_uint((float)c * scale) >> 16;
        }
    }
}

// Slices of two consecutive elements (o points at the first; even offset) as packed BF16 pairs.
__device__ __forceinline__ void store_slices2(__nv_bfloat16* o, int64_t slice_stride, int NS, int64_t F0,
                                              int64_t F1) {
    uint32_t b0[5], b1[5];
    slice_digits(F0, NS, b0);
    slice_digits(F1, NS, b1);
#pragma unroll
    for (int p = 0; p < 5; ++p)
        if (p < NS) *(uint32_t*)(o + p * slice_stride) = b0[p] | (b1[p] << 16);
}

template <int FMT>
__device__ __forceinline__ void load_elem(const void* X, int64_t idx, double& d, float& hi, float& lo) {
    if (FMT == FMT_F64) {
        d = ((const double*)X)[idx];
    } else {
        const float2 p = ((const float2*)X)[idx];
        hi = p.x;
        lo = p.y;
    }
}

// Slicing: one warp per row.  F = round(X 2^(T - e)) is a signed integer with
// |F| <= 2^T, T = B1 + 8 (NS - 1); it is cut into NS balanced digits
// c_0 = round(F / 2^(T - B1)), c_p = round(r_p / 2^(T - B1 - 8p)), the last digit
// taking the remainder, so that |c_p| <= 128 for every p.  Slice p stores
// c_p 2^(-8p), exactly representable in BF16.
template <int FMT>
__global__ void __launch_bounds__(256) slice_rows_kernel(const void* __restrict__ X, int64_t rows, int K, int64_t ld,
                                                         int NS, int Kp, __nv_bfloat16* __restrict__ out,
                                                         int64_t slice_stride, int32_t* __restrict__ exps) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const int64_t base = row * ld;
    int emax = -2000;
    for (int k = lane; k < K; k += 32) {
        double d = 0.0;
        float hi = 0.f, lo = 0.f;
        load_elem<FMT>(X, base + k, d, hi, lo);
        const int ex = FMT == FMT_F64 ? exp_f64(d) : exp_f32(hi);
        emax = max(emax, ex);
    }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    // |X| < 2^(emax + 1); the FP32-pair rounding margin is absorbed because the
    // top digit may reach 2^B1 = 128 exactly.
    const int e = emax <= -2000 ? 0 : emax + 1;
    if (lane == 0) exps[row] = e;
    const int T = SLICE_B1 + 8 * (NS - 1);
    __nv_bfloat16* o0 = out + row * Kp;
    const uint64_t* Xb = (const uint64_t*)X;
    for (int k = 2 * lane; k < Kp; k += 64) {  // two elements per lane (Kp is even)
        int64_t F0 = 0, F1 = 0;
        if (emax > -2000) {
            if (k < K) F0 = fixed_elem<FMT>(Xb[base + k], T - e);
            if (k + 1 < K) F1 = fixed_elem<FMT>(Xb[base + k + 1], T - e);
        }
        store_slices2(o0 + k, slice_stride, NS, F0, F1);
    }
}

// Gather-slicer: the same slicing, reading element (r, k) of the operand at
//   (r / (rd1 rd2)) rs0 + ((r / rd2) % rd1) rs1 + (r % rd2) rs2 + (k / kd) ks0 + (k % kd) ks1,
// so that a permuted view of a tensor is sliced without materialising it.
// Rows with K <= GATHER_SMEM_K are read once into shared memory (one warp per
// row); longer rows are read twice.
struct GatherMap {
    int64_t rd1, rd2, rs0, rs1, rs2;
    int64_t kd, ks0, ks1;
};

constexpr int GATHER_SMEM_K = 1024;  // rows up to this length are read once (8 KB of shared memory per warp)
constexpr int GATHER_WARPS = 8;

__device__ __forceinline__ int64_t gather_off(const GatherMap& g, int64_t r, int k) {
    const int64_t r0 = r / (g.rd1 * g.rd2), r1 = (r / g.rd2) % g.rd1, r2 = r % g.rd2;
    return r0 * g.rs0 + r1 * g.rs1 + r2 * g.rs2 + (int64_t)(k / g.kd) * g.ks0 + (int64_t)(k % g.kd) * g.ks1;
}

template <int FMT>
__global__ void __launch_bounds__(32 * GATHER_WARPS) slice_gather_kernel(const void* __restrict__ X, GatherMap g,
                                                                         int64_t rows, int K, int NS, int Kp,
                                                                         __nv_bfloat16* __restrict__ out,
                                                                         int64_t slice_stride,
                                                                         int32_t* __restrict__ exps) {
    extern __shared__ uint64_t srow_all[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * GATHER_WARPS + wib;
    if (row >= rows) return;
    const bool cached = K <= GATHER_SMEM_K;
    uint64_t* srow = srow_all + (size_t)wib * GATHER_SMEM_K;
    const int64_t rbase = gather_off(g, row, 0);
    int emax = -2000;
    for (int k = lane; k < K; k += 32) {
        const int64_t off = rbase + (int64_t)(k / g.kd) * g.ks0 + (int64_t)(k % g.kd) * g.ks1;
        const uint64_t bits = ((const uint64_t*)X)[off];
        if (cached) srow[k] = bits;
        const int ex = FMT == FMT_F64 ? exp_f64(__longlong_as_double((long long)bits))
                                      : exp_f32(__uint_as_float((uint32_t)(bits & 0xffffffffu)));
        emax = max(emax, ex);
    }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    __syncwarp();
    const int e = emax <= -2000 ? 0 : emax + 1;
    if (lane == 0) exps[row] = e;
    const int T = SLICE_B1 + 8 * (NS - 1);
    __nv_bfloat16* o0 = out + row * Kp;
    const uint64_t* Xb = (const uint64_t*)X;
    auto elem = [&](int k) -> uint64_t {
        return cached ? srow[k] : Xb[rbase + (int64_t)(k / g.kd) * g.ks0 + (int64_t)(k % g.kd) * g.ks1];
    };
    for (int k = 2 * lane; k < Kp; k += 64) {  // two elements per lane (Kp is even)
        int64_t F0 = 0, F1 = 0;
        if (emax > -2000) {
            if (k < K) F0 = fixed_elem<FMT>(elem(k), T - e);
            if (k + 1 < K) F1 = fixed_elem<FMT>(elem(k + 1), T - e);
        }
        store_slices2(o0 + k, slice_stride, NS, F0, F1);
    }
}

// ---------------------------------------------------------------------------
// PTX helpers (tcgen05, TMA, mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr uint32_t WAIT_LIMIT = 1u << 21;  // try_wait rounds before a wait is declared failed

// Bounded wait.  Gives up after WAIT_LIMIT rounds, or as soon as another CTA
// has recorded a failure in the engine's status word (checked every 256 rounds).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int32_t* status) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && *(volatile const int32_t*)status != 0) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 64-byte swizzle: rows of 64 B, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;      // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;               // descriptor version for tcgen05
    d |= (uint64_t)4 << 61;               // SWIZZLE_64B
    return d;
}

// kind::f16 instruction descriptor: BF16 x BF16 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// The GEMM kernel
// ---------------------------------------------------------------------------
constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 32;  // BF16 elements per stage row (64 bytes)
constexpr int UK = 16;  // K per tcgen05.mma (kind::f16)
constexpr int KCB = KCHUNK / BK;  // k-blocks per exactly-accumulated chunk
constexpr int EPI_WARPS = 8;      // two warps per TMEM lane quadrant, 64 columns each
constexpr int THREADS = 64 + 32 * EPI_WARPS;

template <int NS>
struct UmmaCfg {
    static constexpr int A_SLICE = BM * BK * 2;  // bytes of one 128 x 32 BF16 tile
    static constexpr int B_SLICE = BN * BK * 2;
    static constexpr int STAGE = NS * (A_SLICE + B_SLICE);
    static constexpr int STAGES = (200 * 1024) / STAGE >= 4 ? 4 : (200 * 1024) / STAGE;
    static constexpr int SMEM = STAGES * STAGE + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr int TMEM_COLS = 512;  // acc0 | acc1 | acc2 (3 x 128 used)
};

struct UmmaArgs {
    int M, N, Kp;
    int K;           // algorithmic K (before padding), for the flop count
    int prof_class;
    const int32_t* eA;
    const int32_t* eB;
    void* C;
    int64_t ldc;
    int out_fmt;
    int group_m;
    int32_t* status;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// hi + lo += a0 + a1 + a2, with a0, a1 exact (integer-valued) and a2 small:
// two error-free TwoSum steps, the rounding errors folded into lo.
__device__ __forceinline__ void df_accumulate(float& hi, float& lo, float a0, float a1, float a2) {
    const float s = __fadd_rn(hi, a0);
    const float bp = __fsub_rn(s, hi);
    const float e1 = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(a0, bp));
    const float t = __fadd_rn(s, a1);
    const float bq = __fsub_rn(t, s);
    const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bq)), __fsub_rn(a1, bq));
    const float l = __fadd_rn(lo, __fadd_rn(__fadd_rn(e1, e2), a2));
    const float h = __fadd_rn(t, l);  // renormalise (fast two-sum, |t| >= |l|)
    lo = __fsub_rn(l, __fsub_rn(h, t));
    hi = h;
}

template <int NS>
__global__ void __launch_bounds__(THREADS, 1) umma_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, UmmaArgs args) {
    using Cfg = UmmaCfg<NS>;
    constexpr int STAGES = Cfg::STAGES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * Cfg::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* chunk_full = empty + STAGES;
    uint64_t* chunk_empty = chunk_full + 1;
    uint32_t* tmem_slot = (uint32_t*)(chunk_empty + 1);
    int* s_fail = (int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = (args.N + BN - 1) / BN;
    const int m_tiles = (args.M + BM - 1) / BM;
    const int pid = blockIdx.x;
    const int gm = args.group_m;
    const int group = pid / (gm * n_tiles);
    const int first_m = group * gm;
    const int gsize = min(m_tiles - first_m, gm);
    const int tile_m = first_m + (pid % (gm * n_tiles)) % gsize;
    const int tile_n = (pid % (gm * n_tiles)) / gsize;
    const int num_kb = args.Kp / BK;
    const int n_chunks = (num_kb + KCB - 1) / KCB;

    // another CTA already failed: leave (uniformly) before touching TMEM or issuing copies
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = *(volatile const int32_t*)args.status;
    __syncthreads();
    if (s_abort != 0) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(chunk_full, 1);
        mbar_init(chunk_empty, EPI_WARPS);
        *s_fail = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < num_kb; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES) {
                    if (!mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, args.status)) {
                        *s_fail = 1;
                        break;
                    }
                }
                uint8_t* sa = smem + s * Cfg::STAGE;
                uint8_t* sb = sa + NS * Cfg::A_SLICE;
                mbar_arrive_expect_tx(&full[s], Cfg::STAGE);
                tma_load_3d(sa, &tmA, &full[s], kb * BK, tile_m * BM, 0);
                tma_load_3d(sb, &tmB, &full[s], kb * BK, tile_n * BN, 0);
                ++issued;
            }
            // every issued load must have landed before the CTA may exit
            const int first = issued > STAGES ? issued - STAGES : 0;
            for (int kb = first; kb < issued; ++kb)
                if (!mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, args.status)) *s_fail = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, BN);
            const uint32_t acc0 = tmem, acc1 = tmem + BN, acc2 = tmem + 2 * BN;
            bool ok = true;
            for (int kb = 0; kb < num_kb && ok; ++kb) {
                const int s = kb % STAGES;
                const int chunk = kb / KCB;
                const bool chunk_start = (kb % KCB) == 0;
                if (chunk_start && chunk > 0) {
                    // the epilogue must have drained the previous chunk's accumulators
                    if (!mbar_wait(chunk_empty, (chunk - 1) & 1, args.status)) {
                        *s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                if (!mbar_wait(&full[s], (kb / STAGES) & 1, args.status)) {
                    *s_fail = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * Cfg::STAGE);
                const uint32_t sb = sa + NS * Cfg::A_SLICE;
#pragma unroll
                for (int kk = 0; kk < BK / UK; ++kk) {
                    const uint32_t koff = kk * UK * 2;  // bytes along K inside the 64-byte row
                    const uint32_t keep = (chunk_start && kk == 0) ? 0u : 1u;
                    // diagonal 0: exact
                    umma_bf16(acc0, sdesc_sw64(sa + koff), sdesc_sw64(sb + koff), idesc, keep);
                    // diagonal 1: exact
                    umma_bf16(acc1, sdesc_sw64(sa + koff), sdesc_sw64(sb + Cfg::B_SLICE + koff), idesc, keep);
                    umma_bf16(acc1, sdesc_sw64(sa + Cfg::A_SLICE + koff), sdesc_sw64(sb + koff), idesc, 1u);
                    // diagonals >= 2: 2^-16 below the leading term
                    bool first2 = keep == 0u;
#pragma unroll
                    for (int p = 0; p < NS; ++p) {
#pragma unroll
                        for (int q = 0; q < NS; ++q) {
                            if (p + q < 2 || p + q > NS - 1) continue;
                            umma_bf16(acc2, sdesc_sw64(sa + p * Cfg::A_SLICE + koff),
                                      sdesc_sw64(sb + q * Cfg::B_SLICE + koff), idesc, first2 ? 0u : 1u);
                            first2 = false;
                        }
                    }
                }
                umma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                if ((kb % KCB) == KCB - 1 || kb == num_kb - 1) umma_commit(chunk_full);
            }
            if (!ok) umma_commit(chunk_full);  // release the epilogue; s_fail marks the result invalid
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 and 64 columns
        const int quad = warp & 3;
        const int colbase = ((warp - 2) >> 2) * 64;
        const int row_local = quad * 32 + lane;
        const int64_t row = (int64_t)tile_m * BM + row_local;
        float hi[64], lo[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            hi[j] = 0.f;
            lo[j] = 0.f;
        }
        bool alive = true;
        for (int c = 0; c < n_chunks; ++c) {
            alive = __all_sync(0xffffffffu, (alive && mbar_wait(chunk_full, c & 1, args.status)) ? 1 : 0) != 0;
            if (!alive) {
                *s_fail = 1;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                uint32_t r0[8], r1[8], r2[8];
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + colbase + g * 8;
                tmem_ld8(taddr, r0);
                tmem_ld8(taddr + BN, r1);
                tmem_ld8(taddr + 2 * BN, r2);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    df_accumulate(hi[g * 8 + j], lo[g * 8 + j], __uint_as_float(r0[j]), __uint_as_float(r1[j]),
                                  __uint_as_float(r2[j]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(chunk_empty);
        }
        if (alive && row < args.M) {
            const int ea = args.eA[row];
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const int64_t col = (int64_t)tile_n * BN + colbase + j;
                if (col < args.N) {
                    const int sc = ea + args.eB[col] - 2 * SLICE_B1;
                    if (args.out_fmt == FMT_F64)
                        ((double*)args.C)[row * args.ldc + col] = ldexp((double)hi[j] + (double)lo[j], sc);
                    else
                        ((float2*)args.C)[row * args.ldc + col] = make_float2(ldexpf(hi[j], sc), ldexpf(lo[j], sc));
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_fail) atomicExch(args.status, (int)HOTRG_ETIMEOUT);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

// 3D map over slices [NS][rows][Kp] BF16, box {BK, box_rows, NS}
static bool make_map(CUtensorMap* m, const void* base, int NS, int64_t rows, int Kp, int box_rows) {
    PFN_encodeTiled enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)NS};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)NS};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Slice counts of the split forms.  HOTRG_SPLIT_BF16_FAST: 3 slices
// everywhere (23 bits, the FP32 accuracy class).  HOTRG_SPLIT_BF16: by default
// 4 slices (31 bits) for the environments and 5 (39 bits) for the coarse
// contraction; HOTRG_SPLIT_SLICES="env,coarse" (each 3..5) overrides them.
static int ns_for(int prec, bool coarse) {
    static int env_ns = 0, coarse_ns = 0;
    if (env_ns == 0) {
        env_ns = 4;
        coarse_ns = 5;
        const char* v = getenv("HOTRG_SPLIT_SLICES");
        int a = 0, b = 0;
        if (v && sscanf(v, "%d,%d", &a, &b) == 2 && a >= 3 && a <= 5 && b >= 3 && b <= 5) {
            env_ns = a;
            coarse_ns = b;
        }
    }
    if (prec == HOTRG_SPLIT_BF16) return coarse ? coarse_ns : env_ns;
    return 3;
}

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

size_t umma_workspace(int prec, int64_t M, int64_t N, int64_t K) {
    const int NS = 5;
    (void)prec;
    const int64_t Kp = round_up(K, BK);
    const int64_t Mp = round_up(M, BM), Np = round_up(N, BN);
    return (size_t)(NS * (Mp + Np) * Kp * 2 + (Mp + Np) * 4 + 4096);
}

template <int NS>
static hotrg_status launch_umma(hotrg_ctx* ctx, const __nv_bfloat16* As, const __nv_bfloat16* Bs, int M, int N,
                                int Kp, const UmmaArgs& a) {
    using Cfg = UmmaCfg<NS>;
    if (attr_once((const void*)umma_gemm_kernel<NS>, ctx->device))
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(umma_gemm_kernel<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 Cfg::SMEM));
    CUtensorMap mA, mB;
    if (!make_map(&mA, As, NS, M, Kp, BM) || !make_map(&mB, Bs, NS, N, Kp, BN))
        return set_err(ctx, HOTRG_ECUDA, "cuTensorMapEncodeTiled failed");
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int h = prof_begin(ctx);
    umma_gemm_kernel<NS><<<tiles, THREADS, Cfg::SMEM, ctx->stream>>>(mA, mB, a);
    prof_end(ctx, h, a.prof_class, 2.0 * M * N * (double)a.K);
    HOTRG_COUNT(1);
    HOTRG_LAUNCH_CHECK(ctx, "umma_gemm_kernel");
    return HOTRG_OK;
}

// The status word kernels enqueued through ctx report into: the slot of the point being
// enqueued, else the context's own word (made with the context, on its device).
int32_t* umma_status_word(hotrg_ctx* ctx) { return ctx->status_slot ? ctx->status_slot : ctx->status_dev; }

hotrg_status umma_gemm_fmt(hotrg_ctx* ctx, int prec, int M, int N, int K, const void* A, int afmt, int64_t lda,
                           const void* B, int bfmt, int64_t ldb, void* C, int cfmt, int64_t ldc, bool coarse) {
    if (!ctx->tc_ok) return set_err(ctx, HOTRG_ENOTSUP, "tensor-core engine needs sm_103");
    const int NS = ns_for(prec, coarse);
    const int Kp = (int)round_up(K, BK);
    const int64_t Mp = round_up(M, BM), Np = round_up(N, BN);
    __nv_bfloat16* As = (__nv_bfloat16*)ws_alloc(ctx, (size_t)NS * Mp * Kp * 2);
    __nv_bfloat16* Bs = (__nv_bfloat16*)ws_alloc(ctx, (size_t)NS * Np * Kp * 2);
    int32_t* eA = (int32_t*)ws_alloc(ctx, (size_t)Mp * 4);
    int32_t* eB = (int32_t*)ws_alloc(ctx, (size_t)Np * 4);
    if (!As || !Bs || !eA || !eB) return set_err(ctx, HOTRG_ENOMEM, "umma workspace exhausted");
    int32_t* st = umma_status_word(ctx);
    if (!st) return set_err(ctx, HOTRG_ENOMEM, "status word");
    cudaStream_t s = ctx->stream;
    const int rows_per_block = 8;
    const int h_slice = prof_begin(ctx);
    if (afmt == FMT_F64)
        slice_rows_kernel<FMT_F64><<<(M + rows_per_block - 1) / rows_per_block, 256, 0, s>>>(
            A, M, K, lda, NS, Kp, As, (int64_t)M * Kp, eA);
    else
        slice_rows_kernel<FMT_F32PAIR><<<(M + rows_per_block - 1) / rows_per_block, 256, 0, s>>>(
            A, M, K, lda, NS, Kp, As, (int64_t)M * Kp, eA);
    if (bfmt == FMT_F64)
        slice_rows_kernel<FMT_F64><<<(N + rows_per_block - 1) / rows_per_block, 256, 0, s>>>(
            B, N, K, ldb, NS, Kp, Bs, (int64_t)N * Kp, eB);
    else
        slice_rows_kernel<FMT_F32PAIR><<<(N + rows_per_block - 1) / rows_per_block, 256, 0, s>>>(
            B, N, K, ldb, NS, Kp, Bs, (int64_t)N * Kp, eB);
    HOTRG_COUNT(2);
    prof_end(ctx, h_slice, PROF_SLICE, 0.0);
    HOTRG_LAUNCH_CHECK(ctx, "slice_rows_kernel");
    UmmaArgs a;
    a.K = K;
    a.prof_class = coarse ? PROF_GEMM_COARSE : PROF_GEMM_ENV;
    a.M = M;
    a.N = N;
    a.Kp = Kp;
    a.eA = eA;
    a.eB = eB;
    a.C = C;
    a.ldc = ldc;
    a.out_fmt = cfmt;
    a.group_m = 16;
    a.status = st;
    if (NS == 5) return launch_umma<5>(ctx, As, Bs, M, N, Kp, a);
    if (NS == 4) return launch_umma<4>(ctx, As, Bs, M, N, Kp, a);
    return launch_umma<3>(ctx, As, Bs, M, N, Kp, a);
}

// C = A B^T with A and B read through gather maps (both FP64 or FP32-pair).
hotrg_status umma_gemm_gather(hotrg_ctx* ctx, int prec, int M, int N, int K, const void* A, const GatherMap& am,
                              int afmt, const void* B, const GatherMap& bm, int bfmt, void* C, int cfmt, int64_t ldc,
                              bool coarse) {
    if (!ctx->tc_ok) return set_err(ctx, HOTRG_ENOTSUP, "tensor-core engine needs sm_103");
    const int NS = ns_for(prec, coarse);
    const int Kp = (int)round_up(K, BK);
    const int64_t Mp = round_up(M, BM), Np = round_up(N, BN);
    __nv_bfloat16* As = (__nv_bfloat16*)ws_alloc(ctx, (size_t)NS * Mp * Kp * 2);
    __nv_bfloat16* Bs = (__nv_bfloat16*)ws_alloc(ctx, (size_t)NS * Np * Kp * 2);
    int32_t* eA = (int32_t*)ws_alloc(ctx, (size_t)Mp * 4);
    int32_t* eB = (int32_t*)ws_alloc(ctx, (size_t)Np * 4);
    if (!As || !Bs || !eA || !eB) return set_err(ctx, HOTRG_ENOMEM, "umma workspace exhausted");
    int32_t* st = umma_status_word(ctx);
    if (!st) return set_err(ctx, HOTRG_ENOMEM, "status word");
    if (attr_once((const void*)slice_gather_kernel<FMT_F64>, ctx->device)) {
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(slice_gather_kernel<FMT_F64>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 GATHER_WARPS * GATHER_SMEM_K * 8));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(slice_gather_kernel<FMT_F32PAIR>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 GATHER_WARPS * GATHER_SMEM_K * 8));
    }
    cudaStream_t s = ctx->stream;
    const int smem = K <= GATHER_SMEM_K ? GATHER_WARPS * GATHER_SMEM_K * 8 : 0;
    const int h_slice = prof_begin(ctx);
    const int64_t gA = (M + GATHER_WARPS - 1) / GATHER_WARPS, gB = (N + GATHER_WARPS - 1) / GATHER_WARPS;
    if (afmt == FMT_F64)
        slice_gather_kernel<FMT_F64><<<(unsigned)gA, 32 * GATHER_WARPS, smem, s>>>(A, am, M, K, NS, Kp, As,
                                                                                  (int64_t)M * Kp, eA);
    else
        slice_gather_kernel<FMT_F32PAIR><<<(unsigned)gA, 32 * GATHER_WARPS, smem, s>>>(A, am, M, K, NS, Kp, As,
                                                                                      (int64_t)M * Kp, eA);
    if (bfmt == FMT_F64)
        slice_gather_kernel<FMT_F64><<<(unsigned)gB, 32 * GATHER_WARPS, smem, s>>>(B, bm, N, K, NS, Kp, Bs,
                                                                                  (int64_t)N * Kp, eB);
    else
        slice_gather_kernel<FMT_F32PAIR><<<(unsigned)gB, 32 * GATHER_WARPS, smem, s>>>(B, bm, N, K, NS, Kp, Bs,
                                                                                      (int64_t)N * Kp, eB);
    HOTRG_COUNT(2);
    prof_end(ctx, h_slice, PROF_SLICE, 0.0);
    HOTRG_LAUNCH_CHECK(ctx, "slice_gather_kernel");
    UmmaArgs a;
    a.K = K;
    a.prof_class = coarse ? PROF_GEMM_COARSE : PROF_GEMM_ENV;
    a.M = M;
    a.N = N;
    a.Kp = Kp;
    a.eA = eA;
    a.eB = eB;
    a.C = C;
    a.ldc = ldc;
    a.out_fmt = cfmt;
    a.group_m = 16;
    a.status = st;
    if (NS == 5) return launch_umma<5>(ctx, As, Bs, M, N, Kp, a);
    if (NS == 4) return launch_umma<4>(ctx, As, Bs, M, N, Kp, a);
    return launch_umma<3>(ctx, As, Bs, M, N, Kp, a);
}

// Gathered contraction with FP64 operands and output, as used by one HOTRG step.
hotrg_status umma_contract_gather(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, const int64_t* am,
                                  const double* B, const int64_t* bm, double* C, int64_t ldc, bool coarse) {
    GatherMap ga{am[0], am[1], am[2], am[3], am[4], am[5], am[6], am[7]};
    GatherMap gb{bm[0], bm[1], bm[2], bm[3], bm[4], bm[5], bm[6], bm[7]};
    const size_t mark = ctx->ws.used;
    hotrg_status s = umma_gemm_gather(ctx, prec, M, N, K, A, ga, FMT_F64, B, gb, FMT_F64, C, FMT_F64, ldc, coarse);
    ctx->ws.used = mark;
    return s;
}

hotrg_status umma_gemm(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, bool coarse) {
    return umma_gemm_fmt(ctx, prec, M, N, K, A, FMT_F64, lda, B, FMT_F64, ldb, C, FMT_F64, ldc, coarse);
}

hotrg_status umma_contract(hotrg_ctx* ctx, int prec, int M, int N, int K, const double* A, int64_t lda,
                           const double* B, int64_t ldb, double* C, int64_t ldc) {
    return umma_gemm_fmt(ctx, prec, M, N, K, A, FMT_F64, lda, B, FMT_F64, ldb, C, FMT_F64, ldc, true);
}

// ---------------------------------------------------------------------------
// Grouped (block-sparse) contraction: the groups of a BsPlan (one per charge
// value) share one slice buffer per operand, laid out group after group with
// every group padded to 128 rows; row pitch = the K set's size rounded up to
// 32.  Operand element (m, k) of group g is X[rowoff[mbase_g + m] + koff[kbase_g + k]]
// and output element (m, n) goes to C[rowC[mbase_g + m] + colC[nbase_g + n]], plus
// pi[rowP[mbase_g + m] + colP[nbase_g + n]] when the output is in a pair layout.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int group_of_row(const BsGroup* gr, int G, int64_t r, bool b_side) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((b_side ? gr[mid].npad : gr[mid].mpad) <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One warp per padded slice row; rows beyond the plan's padded total leave at once.
// X holds FP64 values (FMT_F64) or exact FP32 pairs hi + lo (FMT_F32PAIR).  Rows
// of up to GROUP_SMEM_K elements are read once (4 KB of shared memory per warp).
// k_contig: the K offsets of every group are consecutive (koff[kbase + k] =
// koff[kbase] + k, the case of an operand in a pair layout), so the values are
// read straight from X without the offset table.
constexpr int GROUP_SMEM_K = 512;
template <int FMT>
__global__ void __launch_bounds__(32 * GATHER_WARPS) slice_grouped_kernel(
    const void* __restrict__ X, const int64_t* __restrict__ rowoff, const int64_t* __restrict__ koff,
    const BsGroup* __restrict__ groups, const BsHeader* __restrict__ hdr, int b_side, int k_contig, int NS, int Kp,
    __nv_bfloat16* __restrict__ out, int64_t slice_stride, int32_t* __restrict__ exps) {
    extern __shared__ uint64_t srow_all[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int G = hdr->G;
    const int64_t rows_total = b_side ? hdr->npad_total : hdr->mpad_total;
    uint64_t* srow = srow_all + (size_t)wib * GROUP_SMEM_K;
    const uint64_t* Xb = (const uint64_t*)X;
    const int T = SLICE_B1 + 8 * (NS - 1);
    const int64_t r = (int64_t)blockIdx.x * GATHER_WARPS + wib;
    if (G == 0 || r >= rows_total) return;
    {
        const int g = group_of_row(groups, G, r, b_side != 0);
        const BsGroup gr = groups[g];
        const int64_t local = r - (b_side ? gr.npad : gr.mpad);
        const int rows = b_side ? gr.N : gr.M;
        const int K = gr.K, Kg = gr.Kp;
        const int64_t* kof = koff + gr.kbase;
        __nv_bfloat16* o0 = out + r * Kp;
        if (local >= rows) {  // padding row of the group's last tile
            if (lane == 0) exps[r] = 0;
            for (int k = lane; k < Kg; k += 32)
                for (int p = 0; p < NS; ++p) o0[p * slice_stride + k] = __float2bfloat16_rn(0.f);
            return;
        }
        // the row's base and, for consecutive K offsets, the first of them (independent loads)
        const int64_t rbase = rowoff[(b_side ? gr.nbase : gr.mbase) + local] + ((k_contig && K > 0) ? kof[0] : 0);
        const bool cached = K <= GROUP_SMEM_K;
        int emax = -2000;
        // four elements per lane in flight
        for (int k0 = lane; k0 < K; k0 += 128) {
            uint64_t v[4];
            if (k_contig) {
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = k0 + 32 * u < K ? Xb[rbase + k0 + 32 * u] : 0;
            } else {
                int64_t o[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) o[u] = k0 + 32 * u < K ? kof[k0 + 32 * u] : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = k0 + 32 * u < K ? Xb[rbase + o[u]] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + 32 * u;
                if (k < K) {
                    if (cached) srow[k] = v[u];
                    const int ex = FMT == FMT_F64 ? exp_f64(__longlong_as_double((long long)v[u]))
                                                  : exp_f32(__uint_as_float((uint32_t)(v[u] & 0xffffffffu)));
                    emax = max(emax, ex);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        __syncwarp();
        const int e = emax <= -2000 ? 0 : emax + 1;
        if (lane == 0) exps[r] = e;
        auto elem = [&](int k) -> uint64_t {
            return cached ? srow[k] : Xb[rbase + (k_contig ? (int64_t)k : kof[k])];
        };
        for (int k = 2 * lane; k < Kg; k += 64) {  // two elements per lane (Kg is even)
            int64_t F0 = 0, F1 = 0;
            if (emax > -2000) {
                if (k < K) F0 = fixed_elem<FMT>(elem(k), T - e);
                if (k + 1 < K) F1 = fixed_elem<FMT>(elem(k + 1), T - e);
            }
            store_slices2(o0 + k, slice_stride, NS, F0, F1);
        }
    }
}

struct GroupArgs {
    const BsGroup* groups;
    const BsHeader* hdr;
    const int32_t* eA;
    const int32_t* eB;
    const int64_t* rowC;
    const int64_t* colC;
    const int32_t* pi;  // null, or the output's pair table with its row / column parts
    const int32_t* rowP;
    const int32_t* colP;
    void* C;
    int32_t* status;
};

// Bounded wait that also gives up when this CTA has already failed.
__device__ __forceinline__ bool mbar_wait_cta(uint64_t* bar, uint32_t parity, const int32_t* status,
                                              const int* s_fail) {
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u &&
            (*(volatile const int32_t*)status != 0 || *(volatile const int*)s_fail != 0))
            return false;
    }
    return false;
}

__device__ __forceinline__ void decode_tile(const BsGroup* gr, int G, int t, int& g, int& tm, int& tn) {
    int lo = 0, hi = G - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gr[mid].tile_base <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    g = lo;
    const int loc = t - gr[g].tile_base;
    tm = loc / gr[g].tiles_n;
    tn = loc % gr[g].tiles_n;
}

// Shared memory of the grouped kernel: the stages plus a 32 x 17 FP64 staging
// tile per epilogue warp, through which the output is written row-contiguous.
// TBN is the tile width (output columns per tile): 128, or 64 for thin charge
// blocks.  The three accumulators of a chunk take 3 TBN TMEM columns; at
// TBN = 64 two such sets fit in the 512 columns, so the MMAs of the next chunk
// (usually the next tile: most blocks' K fits in one chunk) run while the
// epilogue drains the previous one.
template <int NS, int TBN>
struct GroupCfg {
    static constexpr int A_SLICE = BM * BK * 2;
    static constexpr int B_SLICE = TBN * BK * 2;
    static constexpr int SETS = 6 * TBN <= 512 ? 2 : 1;  // TMEM accumulator sets
    static constexpr int COLS = TBN / 2;                  // output columns per epilogue warp
    static constexpr int STAGE = NS * (A_SLICE + B_SLICE);
    static constexpr int STG_LD = 17;
    static constexpr int STG_BYTES = EPI_WARPS * 32 * STG_LD * 8;
    static constexpr int STAGES = (200 * 1024 - STG_BYTES) / STAGE >= 4 ? 4 : (200 * 1024 - STG_BYTES) / STAGE;
    static constexpr int SMEM = STAGES * STAGE + STG_BYTES + 1024 /*align*/ + 256 /*barriers*/;
    static constexpr int TMEM_COLS = 512;
};

// Persistent grouped GEMM: CTA b takes tiles b, b + gridDim.x, ...  The stage,
// k-block and chunk counters run on across tiles, so the epilogue of one
// tile (after its TMEM drain) overlaps the MMAs of the next; chunk ch uses
// TMEM accumulator set ch % SETS.
template <int NS, int OUT, int TBN>
__global__ void __launch_bounds__(THREADS, 1) umma_grouped_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB,
                                                                   GroupArgs args) {
    using Cfg = GroupCfg<NS, TBN>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr int SETS = Cfg::SETS;
    constexpr int COLS = Cfg::COLS;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    double* staging = (double*)(smem + STAGES * Cfg::STAGE);
    uint64_t* full = (uint64_t*)(smem + STAGES * Cfg::STAGE + Cfg::STG_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* chunk_full = empty + STAGES;    // [SETS]
    uint64_t* chunk_empty = chunk_full + 2;   // [SETS]
    uint32_t* tmem_slot = (uint32_t*)(chunk_empty + 2);
    int* s_fail = (int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = args.hdr->G;
    const int total = args.hdr->total_tiles;
    __shared__ int s_abort;
    // the group table, read by every tile's decode (a binary search) and by its epilogue
    __shared__ BsGroup sgr[BS_V];
    if (threadIdx.x == 0) s_abort = *(volatile const int32_t*)args.status;
    for (int i = threadIdx.x; i < G; i += blockDim.x) sgr[i] = args.groups[i];
    __syncthreads();
    if (s_abort != 0 || G == 0 || (int)blockIdx.x >= total) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int c = 0; c < SETS; ++c) {
            mbar_init(&chunk_full[c], 1);
            mbar_init(&chunk_empty[c], EPI_WARPS);
        }
        *s_fail = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                int g, tm, tn;
                decode_tile(sgr, G, t, g, tm, tn);
                const BsGroup& gr = sgr[g];
                const int nkb = gr.Kp / BK;
                const int arow = (int)(gr.mpad + (int64_t)tm * BM), brow = (int)(gr.npad + (int64_t)tn * TBN);
                for (int kb = 0; kb < nkb; ++kb) {
                    const int s = it % STAGES;
                    if (it >= (uint32_t)STAGES &&
                        !mbar_wait_cta(&empty[s], ((it / STAGES) - 1) & 1, args.status, s_fail)) {
                        *s_fail = 1;
                        ok = false;
                        break;
                    }
                    uint8_t* sa = smem + s * Cfg::STAGE;
                    uint8_t* sb = sa + NS * Cfg::A_SLICE;
                    mbar_arrive_expect_tx(&full[s], Cfg::STAGE);
                    tma_load_3d(sa, &tmA, &full[s], kb * BK, arow, 0);
                    tma_load_3d(sb, &tmB, &full[s], kb * BK, brow, 0);
                    ++it;
                }
            }
            // every issued load must have landed before the CTA may exit
            const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0;
            for (uint32_t k = first; k < it; ++k)
                if (!mbar_wait(&full[k % STAGES], (k / STAGES) & 1, args.status)) *s_fail = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(BM, TBN);
            uint32_t acc0 = tmem, acc1 = tmem + TBN, acc2 = tmem + 2 * TBN;
            uint32_t it = 0, ch = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                int g, tm, tn;
                decode_tile(sgr, G, t, g, tm, tn);
                const int nkb = sgr[g].Kp / BK;
                for (int kb = 0; kb < nkb; ++kb) {
                    const int s = it % STAGES;
                    const bool chunk_start = (kb % KCB) == 0;
                    if (chunk_start) {
                        const uint32_t set = ch % SETS;
                        // the set was last used by chunk ch - SETS: wait until the epilogue drained it
                        if (ch >= (uint32_t)SETS) {
                            if (!mbar_wait_cta(&chunk_empty[set], ((ch / SETS) - 1) & 1, args.status, s_fail)) {
                                *s_fail = 1;
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                        }
                        acc0 = tmem + set * 3 * TBN;
                        acc1 = acc0 + TBN;
                        acc2 = acc0 + 2 * TBN;
                    }
                    if (!mbar_wait_cta(&full[s], (it / STAGES) & 1, args.status, s_fail)) {
                        *s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * Cfg::STAGE);
                    const uint32_t sb = sa + NS * Cfg::A_SLICE;
#pragma unroll
                    for (int kk = 0; kk < BK / UK; ++kk) {
                        const uint32_t koff = kk * UK * 2;
                        const uint32_t keep = (chunk_start && kk == 0) ? 0u : 1u;
                        umma_bf16(acc0, sdesc_sw64(sa + koff), sdesc_sw64(sb + koff), idesc, keep);
                        umma_bf16(acc1, sdesc_sw64(sa + koff), sdesc_sw64(sb + Cfg::B_SLICE + koff), idesc, keep);
                        umma_bf16(acc1, sdesc_sw64(sa + Cfg::A_SLICE + koff), sdesc_sw64(sb + koff), idesc, 1u);
                        bool first2 = keep == 0u;
#pragma unroll
                        for (int p = 0; p < NS; ++p) {
#pragma unroll
                            for (int q = 0; q < NS; ++q) {
                                if (p + q < 2 || p + q > NS - 1) continue;
                                umma_bf16(acc2, sdesc_sw64(sa + p * Cfg::A_SLICE + koff),
                                          sdesc_sw64(sb + q * Cfg::B_SLICE + koff), idesc, first2 ? 0u : 1u);
                                first2 = false;
                            }
                        }
                    }
                    umma_commit(&empty[s]);
                    ++it;
                    if ((kb % KCB) == KCB - 1 || kb == nkb - 1) {
                        umma_commit(&chunk_full[ch % SETS]);
                        ++ch;
                    }
                }
            }
            if (!ok)  // release the epilogue; s_fail marks the result invalid
                for (int c = 0; c < SETS; ++c) umma_commit(&chunk_full[c]);
        }
    } else {
        const int quad = warp & 3;
        const int colbase = ((warp - 2) >> 2) * COLS;
        const int row_local = quad * 32 + lane;
        uint32_t ch = 0;
        bool alive = true;
        for (int t = blockIdx.x; t < total && alive; t += gridDim.x) {
            int g, tm, tn;
            decode_tile(sgr, G, t, g, tm, tn);
            const BsGroup& gr = sgr[g];
            const int nchunks = (gr.Kp / BK + KCB - 1) / KCB;
            float hi[COLS], lo[COLS];
#pragma unroll
            for (int j = 0; j < COLS; ++j) {
                hi[j] = 0.f;
                lo[j] = 0.f;
            }
            for (int c = 0; c < nchunks; ++c, ++ch) {
                const uint32_t set = ch % SETS;
                alive = __all_sync(0xffffffffu, (alive && mbar_wait_cta(&chunk_full[set], (ch / SETS) & 1,
                                                                         args.status, s_fail))
                                                    ? 1
                                                    : 0) != 0;
                if (!alive) {
                    *s_fail = 1;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int q = 0; q < COLS / 8; ++q) {
                    uint32_t r0[8], r1[8], r2[8];
                    const uint32_t taddr =
                        tmem + set * 3 * TBN + ((uint32_t)(quad * 32) << 16) + colbase + q * 8;
                    tmem_ld8(taddr, r0);
                    tmem_ld8(taddr + TBN, r1);
                    tmem_ld8(taddr + 2 * TBN, r2);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        df_accumulate(hi[q * 8 + j], lo[q * 8 + j], __uint_as_float(r0[j]), __uint_as_float(r1[j]),
                                      __uint_as_float(r2[j]));
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&chunk_empty[set]);
            }
            if (!alive) break;
            // output: each lane holds one row; 16 columns at a time go through the warp's
            // staging tile so that every store covers two rows x 16 consecutive columns
            const int my_lrow = tm * BM + row_local;
            const int row_ok = my_lrow < gr.M ? 1 : 0;
            const int64_t my_roff = row_ok ? args.rowC[gr.mbase + my_lrow] : 0;
            const int32_t* __restrict__ pi = args.pi;
            const int my_rp = (row_ok && pi) ? args.rowP[gr.mbase + my_lrow] : 0;
            const int my_ea = args.eA[gr.mpad + my_lrow];
            float2* stg = (float2*)(staging + (warp - 2) * (32 * Cfg::STG_LD));
            const int cl = lane & 15;
#pragma unroll
            for (int c0 = 0; c0 < COLS; c0 += 16) {
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) stg[lane * Cfg::STG_LD + jj] = make_float2(hi[c0 + jj], lo[c0 + jj]);
                __syncwarp();
                const int lcol = tn * TBN + colbase + c0 + cl;
                const bool col_ok = lcol < gr.N;
                const int64_t coff = col_ok ? args.colC[gr.nbase + lcol] : 0;
                const int ccp = (col_ok && pi) ? args.colP[gr.nbase + lcol] : 0;
                const int ceb = col_ok ? args.eB[gr.npad + lcol] : 0;
#pragma unroll 4
                for (int r = 0; r < 16; ++r) {
                    const int row = 2 * r + (lane >> 4);
                    const int64_t roff = __shfl_sync(0xffffffffu, my_roff, row);
                    const int ea = __shfl_sync(0xffffffffu, my_ea, row);
                    const int rok = __shfl_sync(0xffffffffu, row_ok, row);
                    const int rp = __shfl_sync(0xffffffffu, my_rp, row);
                    if (rok && col_ok) {
                        const int64_t off = roff + coff + (pi ? (int64_t)__ldg(pi + rp + ccp) : 0);
                        const float2 v = stg[row * Cfg::STG_LD + cl];
                        const int sc = ea + ceb - 2 * SLICE_B1;
                        if (OUT == FMT_F32PAIR) {
                            // exact pair, scaled in FP32 (no FP64 arithmetic in this epilogue): a
                            // product with the normal float 2^sc rounds exactly as ldexpf does
                            float2 o;
                            if (sc >= -126 && sc <= 127) {
                                const float p2 = __int_as_float((sc + 127) << 23);
                                o = make_float2(v.x * p2, v.y * p2);
                            } else {
                                o = make_float2(ldexpf(v.x, sc), ldexpf(v.y, sc));
                            }
                            ((float2*)args.C)[off] = o;
                        } else {
                            // FP64: the power-of-two scale is an add to the exponent field of the
                            // (normal or zero) sum
                            const double d = (double)v.x + (double)v.y;
                            long long b = __double_as_longlong(d);
                            if (b & 0x7ff0000000000000ll) b += (long long)sc << 52;
                            ((double*)args.C)[off] = __longlong_as_double(b);
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *s_fail) atomicExch(args.status, (int)HOTRG_ETIMEOUT);
}

int32_t bs_pitch(int64_t nK, int sym) {
    const int64_t kfull = round_up(nK, BK);
    return (int32_t)((sym == SYM_U1 && kfull > 4096) ? std::max<int64_t>(4096, round_up(kfull / 2, BK)) : kfull);
}

size_t umma_grouped_workspace(int64_t nM, int64_t nK, int64_t nN, int sym) {
    const int64_t Kp = bs_pitch(nK, sym);
    const int64_t rA = round_up(nM, BM) + (int64_t)BS_V * BM, rB = round_up(nN, BN) + (int64_t)BS_V * BN;
    return (size_t)(5 * (rA + rB) * Kp * 2 + (rA + rB) * 4 + 4096);
}

template <int NS, int OUT, int TBN>
static hotrg_status launch_grouped(hotrg_ctx* ctx, const __nv_bfloat16* As, int64_t rA, const __nv_bfloat16* Bs,
                                   int64_t rB, int Kp, const GroupArgs& a, int prof_class) {
    using Cfg = GroupCfg<NS, TBN>;
    if (attr_once((const void*)umma_grouped_kernel<NS, OUT, TBN>, ctx->device))
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(umma_grouped_kernel<NS, OUT, TBN>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM));
    CUtensorMap mA, mB;
    if (!make_map(&mA, As, NS, rA, Kp, BM) || !make_map(&mB, Bs, NS, rB, Kp, TBN))
        return set_err(ctx, HOTRG_ECUDA, "cuTensorMapEncodeTiled failed");
    // persistent grid: one CTA per SM; HOTRG_GROUPED_CTAS (tuning / diagnosis) caps it, leaving SMs
    // to kernels of other worker streams
    static int cap = -1;
    if (cap < 0) {
        const char* v = getenv("HOTRG_GROUPED_CTAS");
        cap = (v && atoi(v) > 0) ? atoi(v) : 0;
    }
    const int ctas = cap > 0 && cap < ctx->sm_count ? cap : ctx->sm_count;
    const int h = prof_begin(ctx);
    umma_grouped_kernel<NS, OUT, TBN><<<ctas, THREADS, Cfg::SMEM, ctx->stream>>>(mA, mB, a);
    prof_end(ctx, h, prof_class, 0.0);  // algorithmic flops are counted on the device by the planner
    HOTRG_COUNT(1);
    HOTRG_LAUNCH_CHECK(ctx, "umma_grouped_kernel");
    return HOTRG_OK;
}

hotrg_status umma_grouped(hotrg_ctx* ctx, int prec, const BsPlan& pl, const void* A, int afmt, const void* B,
                          int bfmt, void* C, int cfmt, int prof_class) {
    if (!ctx->tc_ok) return set_err(ctx, HOTRG_ENOTSUP, "tensor-core engine needs sm_103");
    const int NS = ns_for(prec, prof_class == PROF_GEMM_COARSE);
    const int Kp = pl.kp_cap;  // slice row pitch, a multiple of 32
    const int64_t rA = round_up(pl.nM, BM) + (int64_t)BS_V * BM, rB = round_up(pl.nN, BN) + (int64_t)BS_V * BN;
    __nv_bfloat16* As = (__nv_bfloat16*)ws_alloc(ctx, (size_t)NS * rA * Kp * 2);
    __nv_bfloat16* Bs = (__nv_bfloat16*)ws_alloc(ctx, (size_t)NS * rB * Kp * 2);
    int32_t* eA = (int32_t*)ws_alloc(ctx, (size_t)rA * 4);
    int32_t* eB = (int32_t*)ws_alloc(ctx, (size_t)rB * 4);
    if (!As || !Bs || !eA || !eB) return set_err(ctx, HOTRG_ENOMEM, "umma workspace exhausted");
    int32_t* st = umma_status_word(ctx);
    if (!st) return set_err(ctx, HOTRG_ENOMEM, "status word");
    if (attr_once((const void*)slice_grouped_kernel<FMT_F64>, ctx->device)) {
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(slice_grouped_kernel<FMT_F64>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 GATHER_WARPS * GROUP_SMEM_K * 8));
        HOTRG_CUDA_TRY(ctx, cudaFuncSetAttribute(slice_grouped_kernel<FMT_F32PAIR>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 GATHER_WARPS * GROUP_SMEM_K * 8));
    }
    cudaStream_t s = ctx->stream;
    const int smem = GATHER_WARPS * GROUP_SMEM_K * 8;
    const unsigned gA = (unsigned)((rA + GATHER_WARPS - 1) / GATHER_WARPS);
    const unsigned gB = (unsigned)((rB + GATHER_WARPS - 1) / GATHER_WARPS);
    const int kc = pl.kA_contig ? 1 : 0;
    const int h_slice = prof_begin(ctx);
    if (afmt == FMT_F64)
        slice_grouped_kernel<FMT_F64><<<gA, 32 * GATHER_WARPS, smem, s>>>(A, pl.offM0, pl.offK0, pl.groups, pl.hdr, 0,
                                                                         kc, NS, Kp, As, rA * Kp, eA);
    else
        slice_grouped_kernel<FMT_F32PAIR><<<gA, 32 * GATHER_WARPS, smem, s>>>(A, pl.offM0, pl.offK0, pl.groups,
                                                                             pl.hdr, 0, kc, NS, Kp, As, rA * Kp, eA);
    if (bfmt == FMT_F64)
        slice_grouped_kernel<FMT_F64><<<gB, 32 * GATHER_WARPS, smem, s>>>(B, pl.offN0, pl.offK1, pl.groups, pl.hdr, 1,
                                                                         0, NS, Kp, Bs, rB * Kp, eB);
    else
        slice_grouped_kernel<FMT_F32PAIR><<<gB, 32 * GATHER_WARPS, smem, s>>>(B, pl.offN0, pl.offK1, pl.groups,
                                                                             pl.hdr, 1, 0, NS, Kp, Bs, rB * Kp, eB);
    HOTRG_COUNT(2);
    prof_end(ctx, h_slice, PROF_SLICE, 0.0);
    HOTRG_LAUNCH_CHECK(ctx, "slice_grouped_kernel");
    GroupArgs a;
    a.groups = pl.groups;
    a.hdr = pl.hdr;
    a.eA = eA;
    a.eB = eB;
    a.rowC = pl.offM1;
    a.colC = pl.offN1;
    a.pi = pl.pi_out;
    a.rowP = pl.offM2;
    a.colP = pl.offN2;
    a.C = C;
    a.status = st;
    // the tile width the plan's tile table was made for
    if (pl.tile_n == 64) {
        if (cfmt == FMT_F32PAIR) {
            if (NS == 5) return launch_grouped<5, FMT_F32PAIR, 64>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
            if (NS == 4) return launch_grouped<4, FMT_F32PAIR, 64>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
            return launch_grouped<3, FMT_F32PAIR, 64>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
        }
        if (NS == 5) return launch_grouped<5, FMT_F64, 64>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
        if (NS == 4) return launch_grouped<4, FMT_F64, 64>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
        return launch_grouped<3, FMT_F64, 64>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
    }
    if (pl.tile_n != 128) return set_err(ctx, HOTRG_EINVAL, "grouped tile width must be 64 or 128");
    if (cfmt == FMT_F32PAIR) {
        if (NS == 5) return launch_grouped<5, FMT_F32PAIR, 128>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
        if (NS == 4) return launch_grouped<4, FMT_F32PAIR, 128>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
        return launch_grouped<3, FMT_F32PAIR, 128>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
    }
    if (NS == 5) return launch_grouped<5, FMT_F64, 128>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
    if (NS == 4) return launch_grouped<4, FMT_F64, 128>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
    return launch_grouped<3, FMT_F64, 128>(ctx, As, rA, Bs, rB, Kp, a, prof_class);
}

hotrg_status umma_check_status(hotrg_ctx* ctx) {
    if (!ctx->status_dev) return HOTRG_OK;
    int32_t h = 0;
    HOTRG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->status_dev, 4, cudaMemcpyDeviceToHost, ctx->stream));
    HOTRG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (h != 0) {
        cudaMemsetAsync(ctx->status_dev, 0, 4, ctx->stream);
        return set_err(ctx, (hotrg_status)h,
                       h == HOTRG_ENOTSUP ? "block planner: a product's label sums span more values than its table, "
                                            "or a charge block is wider than the slice pitch"
                                          : "tensor-core engine: a bounded wait ran out");
    }
    return HOTRG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the split contraction (hotrg_contract_noalloc).
//
// For callers that cannot allocate device memory: code that runs while the
// device memory budget belongs to another allocator, or that must not risk
// the implicit device synchronisation of cudaMalloc.  The slices, row
// exponents and the bounded-wait status word live in one file-scope device
// array of NOALLOC_SCRATCH_BYTES; every GPU that loads the library holds it
// until the process exits.  Host code cannot use the array's name as a device
// address: the address comes from cudaGetSymbolAddress, once per device, with
// that device current (done by the first call on each device).  All calls on
// a device share the array, so calls that overlap on the GPU race; the
// status word is cleared by every call, and the slices and exponents are
// fully rewritten by every call.
// ---------------------------------------------------------------------------
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES];

template <int NS>
static hotrg_status noalloc_launch(cudaStream_t st, const __nv_bfloat16* As, const __nv_bfloat16* Bs, int M, int N,
                                   int Kp, const UmmaArgs& a) {
    CUtensorMap mA, mB;
    if (!make_map(&mA, As, NS, M, Kp, BM) || !make_map(&mB, Bs, NS, N, Kp, BN)) return HOTRG_ECUDA;
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    umma_gemm_kernel<NS><<<tiles, THREADS, UmmaCfg<NS>::SMEM, st>>>(mA, mB, a);
    HOTRG_COUNT(1);
    return cudaGetLastError() == cudaSuccess ? HOTRG_OK : HOTRG_ECUDA;
}

static hotrg_status noalloc_setup(int dev) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (g_noalloc_ptr[dev]) return HOTRG_OK;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return HOTRG_ECUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return HOTRG_ENOTSUP;
    if (cudaFuncSetAttribute(umma_gemm_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, UmmaCfg<5>::SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(umma_gemm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, UmmaCfg<4>::SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(umma_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, UmmaCfg<3>::SMEM) !=
            cudaSuccess)
        return HOTRG_ECUDA;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return HOTRG_ECUDA;
    g_noalloc_ptr[dev] = ptr;
    return HOTRG_OK;
}

}  // namespace hotrg

extern "C" hotrg_status hotrg_contract_noalloc(int32_t prec, int32_t M, int32_t N, int32_t K, const double* A,
                                               int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                                               void* cuda_stream) {
    using namespace hotrg;
    if (!A || !B || !C) return HOTRG_EINVAL;
    if (prec != HOTRG_SPLIT_BF16 && prec != HOTRG_SPLIT_BF16_FAST) return HOTRG_EINVAL;
    if (M < 1 || N < 1 || K < 1 || K > 16384 || lda < K || ldb < K || ldc < N) return HOTRG_EINVAL;
    const int NS = ns_for(prec, true);
    const int Kp = (int)round_up(K, BK);
    const int64_t Mp = round_up(M, BM), Np = round_up(N, BN);
    const size_t a_bytes = round_up((int64_t)NS * Mp * Kp * 2, 256), b_bytes = round_up((int64_t)NS * Np * Kp * 2, 256);
    const size_t ea_bytes = round_up(Mp * 4, 256), eb_bytes = round_up(Np * 4, 256);
    if (256 + a_bytes + b_bytes + ea_bytes + eb_bytes > NOALLOC_SCRATCH_BYTES) return HOTRG_EINVAL;  // too large
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return HOTRG_ECUDA;
    }
    hotrg_status s = noalloc_setup(dev);
    if (s != HOTRG_OK) {
        cudaGetLastError();
        return s;
    }
    char* base = (char*)g_noalloc_ptr[dev];
    int32_t* status = (int32_t*)base;  // first 256 bytes: the status word
    __nv_bfloat16* As = (__nv_bfloat16*)(base + 256);
    __nv_bfloat16* Bs = (__nv_bfloat16*)(base + 256 + a_bytes);
    int32_t* eA = (int32_t*)(base + 256 + a_bytes + b_bytes);
    int32_t* eB = (int32_t*)(base + 256 + a_bytes + b_bytes + ea_bytes);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (cudaMemsetAsync(status, 0, 4, st) != cudaSuccess) {
        cudaGetLastError();
        return HOTRG_ECUDA;
    }
    const int rpb = 8;
    slice_rows_kernel<FMT_F64><<<(M + rpb - 1) / rpb, 256, 0, st>>>(A, M, K, lda, NS, Kp, As, (int64_t)M * Kp, eA);
    slice_rows_kernel<FMT_F64><<<(N + rpb - 1) / rpb, 256, 0, st>>>(B, N, K, ldb, NS, Kp, Bs, (int64_t)N * Kp, eB);
    HOTRG_COUNT(2);
    if (cudaGetLastError() != cudaSuccess) return HOTRG_ECUDA;
    UmmaArgs a;
    a.M = M;
    a.N = N;
    a.Kp = Kp;
    a.K = K;
    a.prof_class = PROF_GEMM_OTHER;
    a.eA = eA;
    a.eB = eB;
    a.C = C;
    a.ldc = ldc;
    a.out_fmt = FMT_F64;
    a.group_m = 16;
    a.status = status;
    s = NS == 5 ? noalloc_launch<5>(st, As, Bs, M, N, Kp, a)
                : (NS == 4 ? noalloc_launch<4>(st, As, Bs, M, N, Kp, a) : noalloc_launch<3>(st, As, Bs, M, N, Kp, a));
    if (s != HOTRG_OK) return s;
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return HOTRG_ECUDA;
    }
    return h == 0 ? HOTRG_OK : (hotrg_status)h;
}

namespace hotrg {
}  // namespace hotrg
