// gram_tc.cu -- tcgen05 tensor-core contraction of the fold-grouped Gram in
// split FP16 precision (CV_PREC_FP16X3).
//
// Two kernels.
//
// k_convert (bandwidth-bound, once per element).  The fold-sorted rows are cut
// into k-blocks of 64 rows that never straddle a segment (and so never a
// fold).  For every k-block and every 128-column block of W = [X' | Y' | 1]
// the kernel gathers the rows through the plan's permutation, forms
// v = (x - s_c) * 2^e_c, splits it into an integer part hi = rint(v) (exact in
// FP16 while |hi| <= 2048) and a remainder lo = fp16(v - hi) (|lo| <= 1/2,
// v = hi + lo to within 2^-13), and writes both as the exact shared-memory
// image the tensor core reads: K-major tiles of 128 columns x 64 rows with the
// 128-byte swizzle (column c, row k at byte c * 128 + ((k / 8) ^ (c % 8)) * 16
// + (k % 8) * 2), hi tile then lo tile, 32 KB per (k-block, column block).
// Rows past a segment's end are zero.
//
// k_gram_tc (tensor-bound).  Each (segment, tile) work item forms the
// 128 x 128 tile (bi, bj) of H_S = W_S^T W_S over the segment's rows: Algorithm
// 7 steps 8, 17 and 19 for those rows in one contraction (sums and sums of
// squares sit in the ones column and on the diagonal).  The last column block
// of W is contracted only over its first nlast columns (the used ones rounded
// up to 16): the MMAs of its tiles have N = nlast.  A persistent CTA per
// SM walks items b, b + gridDim.x, ... with three roles:
//   producer thread   per k-block, one bulk copy (cp.async.bulk) of the A
//                     operand's 32 KB and one of B's (none for a diagonal
//                     tile) into a 64 KB stage, completing on `full`;
//   MMA thread        16 tcgen05.mma (kind::f16, M = N = 128, K = 16) per
//                     k-block into two FP32 tensor-memory accumulators
//                       D0 = sum hi*hi            (integer partial sums kept
//                                                  below 2^24 by the choice of
//                                                  scale: exact whatever the
//                                                  accumulator's rounding)
//                       D1 = sum hi*lo + lo*hi + lo*lo   (about 2^-B of D0);
//                     commits release the stage (`empty`) and, after an
//                     item's last k-block, the accumulator set (`acc_full`);
//   epilogue warps    4 warps (one TMEM lane per thread) read D0 and D1,
//                     store D0 exactly as int32 and D1 as float (no FP64
//                     arithmetic, which is slow on this part) and release the
//                     set (`acc_empty`).
// Two accumulator sets (2 x 256 of the 512 TMEM columns) let an item's
// epilogue overlap the next item's MMAs.  Every mbarrier wait is bounded by
// the plan's wait limit: on expiry the waiting thread raises a CTA-wide abort
// flag and all roles leave their loops.  Before the CTA frees its tensor
// memory and exits, the producer waits for the copies it issued to land and
// the MMA thread for its last commit (both bounded by DRAIN_NS, whatever the
// limit), and DEV_ERR_TIMEOUT is recorded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "cvx_internal.cuh"
#include "tc_ptx.cuh"

namespace cvx {
namespace {

constexpr int KB = OPS_KB;                     // rows per k-block: one 128-byte swizzle row of FP16
constexpr int OP_BYTES = TILE * KB * 2;        // one FP16 operand tile (hi or lo): 16 KB
constexpr int STAGES = 3;
constexpr int STAGE_BYTES = 2 * OPS_TILE_BYTES;   // A (hi, lo) and B (hi, lo): 64 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int EPI_WARPS = 4;
constexpr int THREADS = 32 * (2 + EPI_WARPS);  // producer warp, MMA warp, epilogue warps
constexpr int ACC_COLS = 2 * TILE;             // D0 and D1 of one set
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;   // two sets
// Bound of the waits at a role's exit for work it has already issued (bulk
// copies landing in shared memory, MMAs reading it and writing tensor
// memory), whatever the plan's wait limit: the CTA may free its tensor
// memory and exit only once these are done.
constexpr uint64_t DRAIN_NS = 1000000000ull;   // 1 s
constexpr float FP16_OVERFLOW = 65520.0f;            // smallest float that rounds to inf

// ---------------------------------------------------------------------------
// k_convert
// ---------------------------------------------------------------------------
enum ColKind : int { COL_DATA = 0, COL_ONES = 1, COL_ZERO = 2 };

template <typename T>
struct ColSrc {
    const T *ptr;   // column base (row 0), DATA only
    int64_t ld;
    int kind;
    float scale, nshift;       // v = x * scale + nshift  (nshift = -s * scale)
    double scale_d, shift_d;   // for FP64 inputs
};

template <typename T>
__device__ __forceinline__ ColSrc<T> column_source(const PlanView &pl, const T *X, int64_t ldx,
                                                   const T *Y, int64_t ldy, int c) {
    ColSrc<T> cs;
    cs.ptr = X;   // a valid address for every lane
    cs.ld = 0;
    cs.scale = 1.0f;
    cs.nshift = 0.0f;
    cs.scale_d = 1.0;
    cs.shift_d = 0.0;
    if (c < pl.K + pl.M) {
        cs.kind = COL_DATA;
        cs.ptr = c < pl.K ? X + c : Y + (c - pl.K);
        cs.ld = c < pl.K ? ldx : ldy;
        cs.scale = pl.sp.scale_f[c];
        cs.nshift = -pl.sp.shift_f[c] * cs.scale;
        cs.scale_d = (double)cs.scale;
        cs.shift_d = pl.sp.shift[c];
    } else {
        cs.kind = c == pl.K + pl.M ? COL_ONES : COL_ZERO;
    }
    return cs;
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ uint32_t b2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t *>(&h); }

// TF32 value of x (round to nearest, ties away), in an FP32 container.
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// The operand split of each precision, for two consecutive rows:
//   FP16X3: hi = fp16(rint(v)), lo = fp16(v - hi)   (exact integer hi)
//   BF16X3: hi = bf16(v),       lo = bf16(v - hi)
template <int KIND>
struct Split;

template <>
struct Split<KIND_FP16X3> {
    static __device__ __forceinline__ void pair(float a, float b, uint32_t &hi, uint32_t &lo) {
        const __half2 h = __floats2half2_rn(rintf(a), rintf(b));
        const float2 hf = __half22float2(h);
        hi = h2_bits(h);
        lo = h2_bits(__floats2half2_rn(a - hf.x, b - hf.y));
    }
    static __device__ __forceinline__ void pair(double a, double b, uint32_t &hi, uint32_t &lo) {
        const __half ha = __double2half(rint(a)), hb = __double2half(rint(b));
        const __half la = __double2half(a - (double)__half2float(ha));
        const __half lb = __double2half(b - (double)__half2float(hb));
        hi = h2_bits(__halves2half2(ha, hb));
        lo = h2_bits(__halves2half2(la, lb));
    }
};

template <>
struct Split<KIND_BF16X3> {
    static __device__ __forceinline__ void pair(float a, float b, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        hi = b2_bits(h);
        lo = b2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
    }
    static __device__ __forceinline__ void pair(double a, double b, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat16 ha = __double2bfloat16(a), hb = __double2bfloat16(b);
        const __nv_bfloat16 la = __double2bfloat16(a - (double)__bfloat162float(ha));
        const __nv_bfloat16 lb = __double2bfloat16(b - (double)__bfloat162float(hb));
        hi = b2_bits(__halves2bfloat162(ha, hb));
        lo = b2_bits(__halves2bfloat162(la, lb));
    }
};

// Write one column's values for rows 8 rg .. 8 rg + 7 of a k-block into the
// (k-block, column block) operand tile, in the shared-memory image the tensor
// core reads (K-major, 128-byte swizzle, 1024-byte atoms of 8 columns):
//   FP16X3 / BF16X3: the hi tile (16 KB) then the lo tile, column c's 64 rows
//     in one 128-byte row, 16-byte chunk q at (q ^ (c % 8)) * 16;
//   TF32: rows 0..31 then rows 32..63 as two 16 KB tiles, 32 rows of FP32 per
//     128-byte row, chunk q (4 rows) at (q ^ (c % 8)) * 16.
// FP16X3 also tracks the largest |v| (the FP16 range check).
template <int KIND, typename V>
__device__ __forceinline__ void store_column(uint8_t *tile, int c, int rg, const V (&v)[8], float &amax) {
    if constexpr (KIND == KIND_TF32X3) {
        // hi = tf32(v), lo = tf32(v - hi); rows 8 rg .. 8 rg + 7 lie in the
        // 32-row half rg / 4, whose hi tile (16 KB) is followed by its lo tile
        uint32_t hw[8], lw[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float x = (float)v[k];
            hw[k] = tf32_bits(x);
            lw[k] = tf32_bits(x - __uint_as_float(hw[k]));
        }
        uint8_t *base = tile + (rg >> 2) * OPS_TILE_BYTES + c * 128;
        const int q0 = 2 * (rg & 3);
        const uint32_t o0 = ((q0) ^ (c & 7)) << 4, o1 = ((q0 + 1) ^ (c & 7)) << 4;
        *reinterpret_cast<uint4 *>(base + o0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(base + o1) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
        *reinterpret_cast<uint4 *>(base + OP_BYTES + o0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        *reinterpret_cast<uint4 *>(base + OP_BYTES + o1) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
    } else if constexpr (KIND == KIND_TF32) {
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = tf32_bits((float)v[k]);
        uint8_t *base = tile + (rg >> 2) * (OPS_TILE_BYTES / 2) + c * 128;
        const int q0 = 2 * (rg & 3);
        *reinterpret_cast<uint4 *>(base + (((q0) ^ (c & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4 *>(base + (((q0 + 1) ^ (c & 7)) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) Split<KIND>::pair(v[2 * q], v[2 * q + 1], hw[q], lw[q]);
        if constexpr (KIND == KIND_FP16X3) {
#pragma unroll
            for (int k = 0; k < 8; ++k) amax = fmaxf(amax, (float)fabs(v[k]));
        }
        const uint32_t off = (uint32_t)c * 128u + ((uint32_t)(rg ^ (c & 7)) << 4);
        *reinterpret_cast<uint4 *>(tile + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(tile + OP_BYTES + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// 32 bytes in one store (eight 32-bit words).
__device__ __forceinline__ void st_v8(uint8_t *p, const uint32_t (&w)[8]) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                 "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// Two consecutive 16-byte chunks q and q + 1 (q even) of a column's 128-byte
// row, in the row's swizzled order: they land in one aligned 32-byte sector,
// swapped when the column's swizzle phase c % 8 is odd.
__device__ __forceinline__ void store_chunk_pair(uint8_t *row, int c, int q, const uint32_t *lo4, const uint32_t *hi4) {
    const int sw = c & 7;
    const uint32_t w[8] = {sw & 1 ? hi4[0] : lo4[0], sw & 1 ? hi4[1] : lo4[1], sw & 1 ? hi4[2] : lo4[2],
                           sw & 1 ? hi4[3] : lo4[3], sw & 1 ? lo4[0] : hi4[0], sw & 1 ? lo4[1] : hi4[1],
                           sw & 1 ? lo4[2] : hi4[2], sw & 1 ? lo4[3] : hi4[3]};
    st_v8(row + (((q ^ sw) & ~1) << 4), w);
}

// Rows 16 f .. 16 f + 15 of column c of a (k-block, column block) operand
// tile, the same image store_column writes for rows 8 rg .. 8 rg + 7, in
// 32-byte stores (whole sectors, half the store instructions).
template <int KIND>
__device__ __forceinline__ void store_column16(uint8_t *tile, int c, int f, const float (&v)[16], float &amax) {
    if constexpr (KIND == KIND_TF32 || KIND == KIND_TF32X3) {
        uint32_t hw[16], lw[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            hw[k] = tf32_bits(v[k]);
            if constexpr (KIND == KIND_TF32X3) lw[k] = tf32_bits(v[k] - __uint_as_float(hw[k]));
        }
        // the 32-row half f / 2, chunks 4 (f % 2) .. + 3 (four rows each)
        const int q0 = 4 * (f & 1);
        if constexpr (KIND == KIND_TF32) {
            uint8_t *row = tile + (f >> 1) * (OPS_TILE_BYTES / 2) + c * 128;
            store_chunk_pair(row, c, q0, hw, hw + 4);
            store_chunk_pair(row, c, q0 + 2, hw + 8, hw + 12);
        } else {
            uint8_t *row = tile + (f >> 1) * OPS_TILE_BYTES + c * 128;
            store_chunk_pair(row, c, q0, hw, hw + 4);
            store_chunk_pair(row, c, q0 + 2, hw + 8, hw + 12);
            store_chunk_pair(row + OP_BYTES, c, q0, lw, lw + 4);
            store_chunk_pair(row + OP_BYTES, c, q0 + 2, lw + 8, lw + 12);
        }
    } else {
        uint32_t hw[8], lw[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) Split<KIND>::pair(v[2 * q], v[2 * q + 1], hw[q], lw[q]);
        if constexpr (KIND == KIND_FP16X3) {
#pragma unroll
            for (int k = 0; k < 16; ++k) amax = fmaxf(amax, fabsf(v[k]));
        }
        uint8_t *row = tile + c * 128;
        store_chunk_pair(row, c, 2 * f, hw, hw + 4);
        store_chunk_pair(row + OP_BYTES, c, 2 * f, lw, lw + 4);
    }
}

template <typename T>
struct Acc {
    using type = float;
};
template <>
struct Acc<double> {
    using type = double;
};

template <typename T>
__device__ __forceinline__ typename Acc<T>::type prep_value(const ColSrc<T> &cs, T x) {
    return fmaf((float)x, cs.scale, cs.nshift);
}
template <>
__device__ __forceinline__ double prep_value<double>(const ColSrc<double> &cs, double x) {
    return (x - cs.shift_d) * cs.scale_d;
}

// Block of 256 threads per column block cb and a run of its k-blocks
// (g_begin, g_begin + g_step, ... below g_end).  Warp w takes rows 8 w ..
// 8 w + 7 of the k-block (lanes 0..7 fetch their row indices, shared by
// shuffle) and each lane four of the block's columns.  When the whole block
// is X columns and rows are 16-byte aligned (x_vec), lane q takes columns
// 4 q .. 4 q + 3 and loads them as one float4, so a warp load covers 512
// contiguous bytes of a row; otherwise lane q takes columns q, q + 32, q + 64,
// q + 96 with one scalar load each, so each warp load covers 32 contiguous
// elements.  Each thread then writes, for each of its columns, one 16-byte hi
// chunk and one lo chunk (its 8 rows) of the swizzled tiles.
template <typename T, int KIND>
__device__ __forceinline__ void convert_range(const PlanView &pl, const T *__restrict__ X, int64_t ldx,
                                              const T *__restrict__ Y, int64_t ldy, int x_vec, int cb, int g_begin,
                                              int g_end, int g_step) {
    using V = typename Acc<T>::type;
    const int t = threadIdx.x, lane = t & 31, rg = t >> 5;
    const bool vec = sizeof(T) == 4 && x_vec && (cb + 1) * TILE <= pl.K;   // uniform over the block
    const int c0 = vec ? 4 * lane : lane, cstep = vec ? 1 : 32;            // my columns: c0 + j cstep
    const int cg0 = cb * TILE + c0;
    ColSrc<T> cs[4];
    V fill[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        cs[j] = column_source(pl, X, ldx, Y, ldy, cg0 + j * cstep);
        fill[j] = cs[j].kind == COL_ONES ? V(1) : V(0);
    }
    float amax = 0.0f;
    const int k_lane = 8 * rg + lane;
    // software pipeline: the next k-block's record and row indices load while
    // this one's data loads, converts and stores
    int g = g_begin;
    KBlock kb = g < g_end ? pl.kblocks[g] : KBlock{0, 0};
    int32_t my_row = (lane < 8 && k_lane < kb.valid) ? pl.perm[kb.row0 + k_lane] : -1;
    for (; g < g_end; g += g_step) {
        const int g_next = g + g_step;
        const KBlock kb_next = g_next < g_end ? pl.kblocks[g_next] : KBlock{0, 0};
        V v[4][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int32_t n = __shfl_sync(0xffffffffu, my_row, k);
            const int64_t nn = n < 0 ? 0 : n;
            if (vec) {
                const float4 x4 = __ldg(reinterpret_cast<const float4 *>(X + nn * ldx + cg0));
                const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j][k] = n < 0 ? V(0) : prep_value<T>(cs[j], (T)xs[j]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const T x = __ldg(cs[j].ptr + nn * cs[j].ld);
                    const V val = cs[j].kind == COL_DATA ? prep_value<T>(cs[j], x) : fill[j];
                    v[j][k] = n < 0 ? V(0) : val;
                }
            }
        }
        uint8_t *tile = reinterpret_cast<uint8_t *>(pl.ops) + ((int64_t)g * pl.nb + cb) * ops_tile_bytes(KIND);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            store_column<KIND>(tile, c0 + j * cstep, rg, v[j], amax);
            if (j == 0)   // issue the next block's row-index load early
                my_row = (lane < 8 && k_lane < kb_next.valid) ? pl.perm[kb_next.row0 + k_lane] : -1;
        }
    }
    if (amax >= FP16_OVERFLOW) atomicOr(pl.err, DEV_ERR_RANGE);
}

template <typename T, int KIND>
__global__ void __launch_bounds__(256) k_convert(const __grid_constant__ PlanView pl, const T *__restrict__ X,
                                                 int64_t ldx, const T *__restrict__ Y, int64_t ldy, int x_vec) {
    grid_dep_wait();
    grid_dep_launch();
    convert_range<T, KIND>(pl, X, ldx, Y, ldy, x_vec, blockIdx.y, blockIdx.x, pl.nkb, gridDim.x);
}

// Whole rows, for rows that are not 16-byte aligned (K not a multiple of 4,
// or an unaligned X) and for the batched path: a block converts the
// k-blocks [g0, g1) of one plan.  Its work is the pairs (16-row group f of
// k-block g, column c < D) in (g, f, c) order; thread t takes pairs t,
// t + CD_THREADS, ..., so a warp's loads are consecutive columns of one row
// (each row is read as whole sectors, not as 128-column pieces), and writes
// the group's 16 rows of column c as whole 32-byte sectors of the hi and lo
// tiles (store_column16).  Rows past a k-block's valid count are written as
// zero; columns >= D keep the zeros the plan's operand buffer was created
// with.  The arithmetic per element is that of the other converters.
constexpr int CD_THREADS = 512;


template <int KIND>
__device__ __forceinline__ void convert_pairs(const PlanView &pl, const float *__restrict__ X, int64_t ldx,
                                              const float *__restrict__ Y, int64_t ldy, int g0, int g1) {
    // the block's row indices, k-block by k-block (rows past a k-block's
    // valid count: -1)
    __shared__ int32_t rows_s[CD_MAX_RUN * KB];
    const int K = pl.K, KM = pl.K + pl.M, D = pl.D;
    for (int i = threadIdx.x; i < (g1 - g0) * KB; i += CD_THREADS) {
        const KBlock kb = pl.kblocks[g0 + i / KB];
        const int r = i % KB;
        rows_s[i] = r < kb.valid ? pl.perm[kb.row0 + r] : -1;
    }
    __syncthreads();
    const uint32_t ud = (uint32_t)D;
    const uint32_t pairs = (uint32_t)(g1 - g0) * (KB / 16) * ud;
    float amax = 0.0f;
    for (uint32_t e = threadIdx.x; e < pairs; e += CD_THREADS) {
        const uint32_t gf = e / ud;
        const int c = (int)(e - gf * ud);
        const int f = (int)(gf % (KB / 16)), gl = (int)(gf / (KB / 16));   // group, k-block of the run
        const float *src = c < K ? X + c : Y + (c - K);
        const int64_t ld = c < K ? ldx : ldy;
        const bool data = c < KM;
        const float sc = data ? pl.sp.scale_f[c] : 0.0f;
        const float ns = data ? -pl.sp.shift_f[c] * sc : 1.0f;   // the ones column: 0 * 0 + 1
        const int32_t *rows = rows_s + gl * KB + 16 * f;
        float v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int32_t n = rows[r];
            v[r] = (n >= 0 && data) ? src[(int64_t)n * ld] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = rows[r] >= 0 ? fmaf(v[r], sc, ns) : 0.0f;
        uint8_t *tile =
            reinterpret_cast<uint8_t *>(pl.ops) + ((int64_t)(g0 + gl) * pl.nb + c / TILE) * ops_tile_bytes(KIND);
        store_column16<KIND>(tile, c % TILE, f, v, amax);
    }
    if (amax >= FP16_OVERFLOW) atomicOr(pl.err, DEV_ERR_RANGE);
}

// One plan: block b converts k-blocks [b run, (b + 1) run).
template <int KIND>
__global__ void __launch_bounds__(CD_THREADS, 2) k_convert_direct(const __grid_constant__ PlanView pl,
                                                                 const float *__restrict__ X, int64_t ldx,
                                                                 const float *__restrict__ Y, int64_t ldy, int run) {
    grid_dep_wait();
    grid_dep_launch();
    const int g0 = (int)blockIdx.x * run;
    convert_pairs<KIND>(pl, X, ldx, Y, ldy, g0, min(pl.nkb, g0 + run));
}

// Batched: block per unit (problem, k-blocks [begin, end)).
template <int KIND>
__global__ void __launch_bounds__(CD_THREADS, 2) k_convert_batched(const __grid_constant__ BatchTables bt,
                                                                  const __grid_constant__ BatchArgs ba) {
    grid_dep_wait();
    grid_dep_launch();
    const int4 u = bt.conv_units[blockIdx.x];
    const ProblemArgs &a = batch_arg(bt, ba, u.x);
    convert_pairs<KIND>(bt.views[u.x], (const float *)a.X, a.ldx, (const float *)a.Y, a.ldy, u.y, u.z);
}

// ---------------------------------------------------------------------------
// k_convert_bulk: the same conversion fed by the tensor memory accelerator.
// A producer warp lands each (k-block, column block)'s raw FP32 rows in a
// shared-memory ring, so the data in flight is bounded by the ring, not by
// registers:
//   * rows consecutive in memory (contiguous folds): one 2D tensor copy of a
//     128-column x 64-row box of X (columns past K read as zero) and, for
//     blocks that hold Y columns, one box of the packed Yp = [Y | 1 | 0 ..];
//   * gathered rows: one bulk copy (cp.async.bulk) per row of each part.
// Stage layout: X part [64][128] floats, then Y part [64][ybw] floats.  CTA b
// takes k-blocks g = b, b + gridDim.x, ... and every column block of each in
// turn; the next k-block's record and row indices load while this one's
// copies are issued.  Requires FP32 X with 16-byte aligned rows and
// K % 4 == 0 (so every segment and offset is a multiple of 16 bytes).
// ---------------------------------------------------------------------------
constexpr int CB_MAX_STAGES = 6;
constexpr int CB_XBYTES = KB * TILE * 4;        // 64 rows x 128 FP32: 32 KB
constexpr int CB_THREADS = 32 + 256;            // producer warp + 8 converter warps

struct ConvShared {
    uint64_t full[CB_MAX_STAGES];
    uint64_t empty[CB_MAX_STAGES];
    uint64_t wait_ns;
    volatile int abort_flag;
};

// At a producer's exit: wait (bounded by DRAIN_NS) until the copies of its
// last `issued` stage fills have landed, one fill per stage at most being
// outstanding.  Fill j of a ring of `stages` completes phase j / stages of
// full[j % stages].
__device__ __forceinline__ void drain_fills(uint64_t *full, int stages, uint32_t issued) {
    const uint32_t first = issued > (uint32_t)stages ? issued - (uint32_t)stages : 0u;
    for (uint32_t j = first; j < issued; ++j)
        ptx::mbar_wait_bounded(ptx::smem_u32(&full[j % stages]), (j / stages) & 1u, DRAIN_NS);
}

struct ConvGeom {
    int stages, stage_bytes, ybw, mp;
};

__device__ __forceinline__ bool cb_wait(uint64_t *bar, uint32_t parity, ConvShared &sh) {
    const uint32_t a = ptx::smem_u32(bar);
    if (ptx::mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (true) {
        if (ptx::mbar_try_wait(a, parity)) return true;
        if (sh.abort_flag) return false;
        if (ptx::globaltimer_ns() - t0 > sh.wait_ns) {
            sh.abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void cb_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ptx::smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void cb_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(CB_THREADS, 1)
    k_convert_bulk(PlanView pl, const float *__restrict__ X, int64_t ldx, const float *__restrict__ Yp, ConvGeom geo,
                   const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_y) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ ConvShared sh;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = pl.K, nb = pl.nb, mp = geo.mp, ybw = geo.ybw, stages = geo.stages;
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            ptx::mbar_init(ptx::smem_u32(&sh.full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&sh.empty[s]), 256);
        }
        sh.wait_ns = pl.wait_ns;
        sh.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    grid_dep_wait();
    grid_dep_launch();
    if (warp == 0) {
        // ---------------------------------------------------------- producer
        uint32_t it = 0;
        int g = blockIdx.x;
        KBlock kb = g < pl.nkb ? pl.kblocks[g] : KBlock{0, 0};
        int32_t r_a = lane < kb.valid ? pl.perm[kb.row0 + lane] : -1;
        int32_t r_b = lane + 32 < kb.valid ? pl.perm[kb.row0 + 32 + lane] : -1;
        bool ok = true;
        for (; g < pl.nkb && ok; g += gridDim.x) {
            const int g_next = g + gridDim.x;
            const KBlock kb_next = g_next < pl.nkb ? pl.kblocks[g_next] : KBlock{0, 0};
            const int32_t first = __shfl_sync(0xffffffffu, r_a, 0);
            const bool contig = __all_sync(0xffffffffu, (r_a < 0 || r_a == first + lane) &&
                                                            (r_b < 0 || r_b == first + 32 + lane));
            int32_t n_a = -1, n_b = -1;
            for (int cb = 0; cb < nb; ++cb, ++it) {
                const int c0 = cb * TILE;
                const int xc = c0 < K ? min(TILE, K - c0) : 0;       // X columns of the block
                const bool need_y = c0 + TILE > K;                  // the block holds Y columns
                const int s = it % stages;
                if (it >= (uint32_t)stages && lane == 0) ok = cb_wait(&sh.empty[s], ((it / stages) - 1) & 1, sh);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok || sh.abort_flag) {
                    ok = false;
                    break;
                }
                const uint32_t st = ptx::smem_u32(smem + (size_t)s * geo.stage_bytes);
                const uint32_t sty = st + CB_XBYTES;
                const uint32_t bar = ptx::smem_u32(&sh.full[s]);
                if (contig) {
                    if (lane == 0) {
                        cb_expect_tx(&sh.full[s], (xc > 0 ? (uint32_t)CB_XBYTES : 0u) +
                                                      (need_y ? (uint32_t)KB * ybw * 4u : 0u));
                        if (xc > 0) tma_2d(st, &tm_x, c0, first, bar);
                        if (need_y) tma_2d(sty, &tm_y, 0, first, bar);
                    }
                } else {
                    if (lane == 0)
                        cb_expect_tx(&sh.full[s], (uint32_t)kb.valid * (xc * 4u + (need_y ? (uint32_t)mp * 4u : 0u)));
                    __syncwarp();
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int32_t r = half ? r_b : r_a;
                        const int k = lane + 32 * half;
                        if (r >= 0) {
                            if (xc > 0) bulk_g2s(st + k * TILE * 4, X + (int64_t)r * ldx + c0, xc * 4, bar);
                            if (need_y) bulk_g2s(sty + k * ybw * 4, Yp + (int64_t)r * mp, mp * 4, bar);
                        }
                    }
                }
                if (cb == 0) {
                    n_a = lane < kb_next.valid ? pl.perm[kb_next.row0 + lane] : -1;
                    n_b = lane + 32 < kb_next.valid ? pl.perm[kb_next.row0 + 32 + lane] : -1;
                }
            }
            kb = kb_next;
            r_a = n_a;
            r_b = n_b;
        }
        // on an abort, copies already issued may still be landing in the ring
        if (lane == 0) drain_fills(sh.full, stages, it);
    } else {
        // -------------------------------------------------------- converters
        // warp w owns columns 16 w .. 16 w + 15 over all 64 rows; lane l takes
        // the four columns 16 w + 4 (l % 4) .. + 3 and rows 8 (l / 4) .. + 7, so
        // that each store instruction writes 4 complete 128-byte tile rows
        const int t = tid - 32, cw = t >> 5;
        const int rg = lane >> 2;                   // rows 8 rg .. 8 rg + 7 (the tile chunk)
        const int c0 = 16 * cw + 4 * (lane & 3);    // columns c0 .. c0 + 3
        float amax = 0.0f;
        uint32_t it = 0;
        bool ok = true;
        for (int g = blockIdx.x; g < pl.nkb && ok; g += gridDim.x) {
            const KBlock kb = pl.kblocks[g];
            for (int cb = 0; cb < nb; ++cb, ++it) {
                const int s = it % stages;
                const int cg0 = cb * TILE + c0;
                // quad source: X part, Y part, or zero (K % 4 == 0: a quad never straddles)
                const bool in_x = cg0 < K;
                const bool in_y = !in_x && cg0 - K + 3 < ybw;
                float sc[4], ns[4];
                bool live[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int cg = cg0 + j;
                    live[j] = cg < pl.D && (in_x || in_y);
                    sc[j] = live[j] && cg < pl.K + pl.M ? pl.sp.scale_f[cg] : 1.0f;
                    ns[j] = live[j] && cg < pl.K + pl.M ? -pl.sp.shift_f[cg] * sc[j] : 0.0f;
                }
                if (!cb_wait(&sh.full[s], (it / stages) & 1, sh)) {
                    ok = false;
                    break;
                }
                if (cb == nb - 1 && 16 * cw >= pl.nlast) {
                    // columns the contraction never reads (zeroed at plan time)
                    cb_arrive(&sh.empty[s]);
                    continue;
                }
                const uint8_t *stage = smem + (size_t)s * geo.stage_bytes;
                const float *src = in_x ? reinterpret_cast<const float *>(stage) + c0
                                        : reinterpret_cast<const float *>(stage + CB_XBYTES) + (in_y ? cg0 - K : 0);
                const int pitch = in_x ? TILE : ybw;
                float v[4][8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int row = 8 * rg + k;
                    const float4 x4 = *reinterpret_cast<const float4 *>(src + row * pitch);
                    const float xs[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        v[j][k] = (row < kb.valid && live[j]) ? fmaf(xs[j], sc[j], ns[j]) : 0.0f;
                }
                cb_arrive(&sh.empty[s]);   // raw values are in registers now
                uint8_t *tile = reinterpret_cast<uint8_t *>(pl.ops) + ((int64_t)g * nb + cb) * ops_tile_bytes(KIND);
#pragma unroll
                for (int j = 0; j < 4; ++j) store_column<KIND>(tile, c0 + j, rg, v[j], amax);
            }
        }
        if (amax >= FP16_OVERFLOW) atomicOr(pl.err, DEV_ERR_RANGE);
    }
    __syncthreads();
    if (tid == 0 && sh.abort_flag) atomicOr(pl.err, DEV_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------
// k_convert_rows: the conversion for gathered rows (folds that are not
// contiguous row ranges, e.g. random folds).  The bulk converter above copies
// each (k-block, column block) as 64 row pieces of 512 bytes, one copy
// request each; with gathered rows that reached 3.7 TB/s against 6.6 TB/s
// for contiguous folds on N = 1e6, K = 1024.  Here a ring fill is R whole
// rows (R = 16, or 8 for wide rows): per row one copy of its K floats of X
// and one of its mp floats of Yp = [Y | 1 | 0 ..], so a k-block takes
// 2 x 64 requests whatever the number of column blocks.  Stage layout: X
// part [R][K] floats, then the Y part [R][mp].  Converter thread t takes
// columns t, t + 512, ... < D of every fill and writes, for each, the fill's
// 16 rows of the column's hi and lo tiles as whole 32-byte sectors, one
// 256-bit store each (with 16-byte stores the L2 tag lookups limited the
// kernel: 44-69 % of their peak in ncu).  The arithmetic per element is that
// of the other converters.
// ---------------------------------------------------------------------------
constexpr int CR_CONV = 512;               // converter threads (16 warps)
constexpr int CR_THREADS = 32 + CR_CONV;    // producer warp + converters
constexpr int CR_MAX_COLS = 3;              // columns per converter thread: D <= 1536

struct RowGeom {
    int rows;          // R, rows per fill: 16 or 8
    int stages;
    int stage_bytes;   // a multiple of 1024
    int mp;            // floats per packed Y row
    int xbytes;        // R * K * 4: the X part of a stage
};

template <int KIND, int R>
__global__ void __launch_bounds__(CR_THREADS, 1)
    k_convert_rows(PlanView pl, const float *__restrict__ X, int64_t ldx, const float *__restrict__ Yp, RowGeom geo) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ ConvShared sh;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = pl.K, mp = geo.mp, stages = geo.stages;
    constexpr int fills = KB / R;   // ring fills per k-block
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) {
            ptx::mbar_init(ptx::smem_u32(&sh.full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&sh.empty[s]), CR_CONV);
        }
        sh.wait_ns = pl.wait_ns;
        sh.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    grid_dep_wait();
    grid_dep_launch();
    if (warp == 0) {
        // ---------------------------------------------------------- producer
        uint32_t it = 0;
        bool ok = true;
        for (int g = blockIdx.x; g < pl.nkb && ok; g += gridDim.x) {
            const KBlock kb = pl.kblocks[g];
            const int32_t r_a = lane < kb.valid ? pl.perm[kb.row0 + lane] : -1;
            const int32_t r_b = lane + 32 < kb.valid ? pl.perm[kb.row0 + 32 + lane] : -1;
            for (int f = 0; f < fills; ++f, ++it) {
                const int s = it % stages;
                if (it >= (uint32_t)stages && lane == 0) ok = cb_wait(&sh.empty[s], ((it / stages) - 1) & 1, sh);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok || sh.abort_flag) {
                    ok = false;
                    break;
                }
                const int k0 = f * R;
                const int nv = max(0, min(R, kb.valid - k0));   // rows of the fill in use
                const int k = k0 + lane;                        // this lane's row of the k-block
                const int32_t ra = __shfl_sync(0xffffffffu, r_a, k & 31);
                const int32_t rb = __shfl_sync(0xffffffffu, r_b, k & 31);
                const int32_t row = k < 32 ? ra : rb;
                const uint32_t st = ptx::smem_u32(smem + (size_t)s * geo.stage_bytes);
                const uint32_t bar = ptx::smem_u32(&sh.full[s]);
                if (lane == 0) cb_expect_tx(&sh.full[s], (uint32_t)nv * (uint32_t)(K + mp) * 4u);
                __syncwarp();
                if (lane < nv) {
                    bulk_g2s(st + (uint32_t)(lane * K * 4), X + (int64_t)row * ldx, (uint32_t)K * 4u, bar);
                    bulk_g2s(st + (uint32_t)(geo.xbytes + lane * mp * 4), Yp + (int64_t)row * mp, (uint32_t)mp * 4u,
                             bar);
                }
            }
        }
        // on an abort, copies already issued may still be landing in the ring
        if (lane == 0) drain_fills(sh.full, stages, it);
    } else {
        // -------------------------------------------------------- converters
        const int t = tid - 32;
        const int D = pl.D;
        float sc[CR_MAX_COLS], ns[CR_MAX_COLS];
#pragma unroll
        for (int j = 0; j < CR_MAX_COLS; ++j) {
            const int c = t + CR_CONV * j;
            const bool data = c < pl.K + pl.M;
            sc[j] = data ? pl.sp.scale_f[c] : 1.0f;            // the ones column: 1 * 1 + 0
            ns[j] = data ? -pl.sp.shift_f[c] * sc[j] : 0.0f;
        }
        float amax = 0.0f;
        uint32_t it = 0;
        bool ok = true;
        for (int g = blockIdx.x; g < pl.nkb && ok; g += gridDim.x) {
            const KBlock kb = pl.kblocks[g];
            uint8_t *tiles = reinterpret_cast<uint8_t *>(pl.ops) + (int64_t)g * pl.nb * ops_tile_bytes(KIND);
            for (int f = 0; f < fills; ++f, ++it) {
                const int s = it % stages;
                if (!cb_wait(&sh.full[s], (it / stages) & 1, sh)) {
                    ok = false;
                    break;
                }
                const float *xs = reinterpret_cast<const float *>(smem + (size_t)s * geo.stage_bytes);
                const float *ys = reinterpret_cast<const float *>(smem + (size_t)s * geo.stage_bytes + geo.xbytes);
                const int k0 = f * R;
                const int nv = max(0, min(R, kb.valid - k0));
#pragma unroll
                for (int j = 0; j < CR_MAX_COLS; ++j) {
                    const int c = t + CR_CONV * j;
                    if (c < D) {
                        const float *src = c < K ? xs + c : ys + (c - K);
                        const int pitch = c < K ? K : mp;
                        uint8_t *tile = tiles + (int64_t)(c / TILE) * ops_tile_bytes(KIND);
                        if constexpr (R == 16) {
                            float v[16];
#pragma unroll
                            for (int r = 0; r < 16; ++r) v[r] = r < nv ? fmaf(src[r * pitch], sc[j], ns[j]) : 0.0f;
                            store_column16<KIND>(tile, c % TILE, k0 >> 4, v, amax);
                        } else {
                            float v[8];
#pragma unroll
                            for (int r = 0; r < 8; ++r) v[r] = r < nv ? fmaf(src[r * pitch], sc[j], ns[j]) : 0.0f;
                            store_column<KIND>(tile, c % TILE, k0 >> 3, v, amax);
                        }
                    }
                }
                cb_arrive(&sh.empty[s]);
            }
        }
        if (amax >= FP16_OVERFLOW) atomicOr(pl.err, DEV_ERR_RANGE);
    }
    __syncthreads();
    if (tid == 0 && sh.abort_flag) atomicOr(pl.err, DEV_ERR_TIMEOUT);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2D FP32 tensor map: `width` columns x `rows` rows, leading dimension ld
// floats, box of box_w x box_h; reads outside the tensor are zero.
bool make_map_f32(CUtensorMap *map, const void *ptr, int64_t width, int64_t rows, int64_t ld, int box_w,
                  int box_h) {
    auto encode = tensor_map_encoder();
    if (!encode) return false;
    cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// k_gram_tc
// ---------------------------------------------------------------------------
struct GramShared {
    uint64_t full[STAGES];       // producer -> MMA: operands landed (bulk-copy complete_tx)
    uint64_t empty[STAGES];      // MMA -> producer: stage consumed (tcgen05.commit)
    uint64_t acc_full[2];        // MMA -> epilogue: accumulator set final (tcgen05.commit)
    uint64_t acc_empty[2];       // epilogue -> MMA: set drained (count = 32 * EPI_WARPS)
    uint32_t tmem_slot;
    uint64_t wait_ns;
    volatile int abort_flag;
};

// Bounded wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, GramShared &sh) {
    const uint32_t a = ptx::smem_u32(bar);
    if (ptx::mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (true) {
        if (ptx::mbar_try_wait(a, parity)) return true;
        if (sh.abort_flag) return false;
        if (ptx::globaltimer_ns() - t0 > sh.wait_ns) {
            sh.abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ptx::smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(bar)
                 : "memory");
}

// One work item as the roles need it: its operand k-blocks, tile and partial.
struct ItemGeo {
    const uint8_t *ops;
    int32_t nb, g0, g1;
    int32_t nw;           // columns of block bj the item computes: TILE, or nlast for the last block
    TileCoord tc;
    int32_t *out_hi;
    float *out_lo;
};

__device__ __forceinline__ ItemGeo item_geo(const PlanView &pl, int64_t item) {
    ItemGeo ig;
    const int seg = (int)(item / pl.ntiles);
    ig.ops = reinterpret_cast<const uint8_t *>(pl.ops);
    ig.nb = pl.nb;
    ig.g0 = pl.seg_kb[seg];
    ig.g1 = pl.seg_kb[seg + 1];
    ig.tc = pl.tiles[item % pl.ntiles];
    ig.nw = ig.tc.bj == pl.nb - 1 ? pl.nlast : TILE;
    ig.out_hi = part_hi(pl) + item * TILE_ELEMS;
    ig.out_lo = part_lo(pl) + item * TILE_ELEMS;
    return ig;
}

// The work items of this CTA: items b, b + gridDim.x, ... of one plan, or a
// batched launch's list for this CTA (problem, item) over many plans.
template <bool BATCHED>
struct ItemSource {
    const PlanView *pl;
    const BatchTables *bt;
    int64_t begin, end, step;
    __device__ __forceinline__ ItemSource(const PlanView &p, const BatchTables &b) : pl(&p), bt(&b) {
        if constexpr (BATCHED) {
            begin = b.gram_cta[blockIdx.x];
            end = b.gram_cta[blockIdx.x + 1];
            step = 1;
        } else {
            begin = blockIdx.x;
            end = (int64_t)p.nsegs * p.ntiles;
            step = gridDim.x;
        }
    }
    __device__ __forceinline__ ItemGeo operator()(int64_t idx) const {
        if constexpr (BATCHED) {
            const int2 e = bt->gram_items[idx];
            return item_geo(bt->views[e.x], e.y);
        } else {
            return item_geo(*pl, idx);
        }
    }
};

// The MMAs of one ring fill (a k-block, or for TF32X3 a 32-row half) of an
// item whose block bj has NW columns, into D0 = d0 and D1 = d0 + NW.  The
// stage holds A at a_hi (hi part, then its lo part 16 KB on) and, unless the
// tile is diagonal (B = A), B 32 KB on: [hi_B ; lo_B] with lo_B NW rows after
// hi_B.  acc0: the item's D0 / D1 already hold earlier fills.  Widths and
// instruction descriptors are compile-time constants: with them in registers
// the issue loop measured 43 % slower on the bench workload.
template <int KIND, int NW, bool DIAG>
__device__ __forceinline__ void mma_fill(uint32_t d0, uint32_t a_hi, bool acc0) {
    constexpr uint32_t FMT =
        KIND == KIND_FP16X3 ? ptx::FMT_F16 : KIND == KIND_BF16X3 ? ptx::FMT_BF16 : ptx::FMT_TF32;   // TF32, TF32X3
    constexpr uint32_t IDESC = ptx::idesc_f32acc(TILE, NW, FMT);
    // N = 2 NW: B = the hi part and the lo part that follows it, one operand,
    // so A is read once for hi * hi and hi * lo
    constexpr uint32_t IDESC_W = ptx::idesc_f32acc(TILE, 2 * NW, FMT);
    // on a narrow diagonal tile B's lo part is A's, 16 KB after its hi part
    // rather than NW rows after: separate products
    constexpr bool SPLIT_B = DIAG && NW < TILE;
    const uint32_t d1 = d0 + NW;
    const uint32_t a_lo = a_hi + OP_BYTES;
    const uint32_t b_hi = DIAG ? a_hi : a_hi + OPS_TILE_BYTES;
    const uint32_t b_lo = DIAG ? a_lo : b_hi + NW * 128u;
    if constexpr (KIND == KIND_TF32) {
        // two 16 KB halves of 32 rows; 8 TF32 along K = 32 bytes per MMA
#pragma unroll
        for (int kk = 0; kk < KB / 8; ++kk) {
            const uint32_t o = (kk >> 2) * (OPS_TILE_BYTES / 2) + (kk & 3) * 32;
            const uint32_t acc = (acc0 || kk > 0) ? 1u : 0u;
            ptx::mma_tf32_ss(d1, ptx::desc_kmajor_sw128(a_hi + o), ptx::desc_kmajor_sw128(b_hi + o), IDESC, acc);
        }
    } else {
        // FP16 / BF16: 16 values along K = 32 bytes per MMA over a 64-row
        // k-block; TF32X3: 8 values along K = 32 bytes over a 32-row half
#pragma unroll
        for (int kk = 0; kk < KB / 16; ++kk) {
            const uint32_t o = kk * 32;
            const uint32_t acc = (acc0 || kk > 0) ? 1u : 0u;
            const uint64_t ah = ptx::desc_kmajor_sw128(a_hi + o), al = ptx::desc_kmajor_sw128(a_lo + o);
            const uint64_t bh = ptx::desc_kmajor_sw128(b_hi + o), bl = ptx::desc_kmajor_sw128(b_lo + o);
            if constexpr (KIND == KIND_TF32X3) {
                if constexpr (!SPLIT_B) {
                    ptx::mma_tf32_ss(d0, ah, bh, IDESC_W, acc);   // [D0 | D1] = hi_A [hi_B ; lo_B]
                } else {
                    ptx::mma_tf32_ss(d0, ah, bh, IDESC, acc);     // D0 += hi*hi
                    ptx::mma_tf32_ss(d1, ah, bl, IDESC, acc);     // D1 += hi*lo
                }
                ptx::mma_tf32_ss(d1, al, bh, IDESC, 1u);          // D1 += lo*hi (lo*lo dropped)
            } else {
                if constexpr (!SPLIT_B) {
                    // [D0 | D1] (+)= hi_A [hi_B ; lo_B]: D0 += hi*hi, D1 += hi*lo
                    ptx::mma_f16_ss(d0, ah, bh, IDESC_W, acc);
                } else {
                    ptx::mma_f16_ss(d0, ah, bh, IDESC, acc);     // D0 += hi*hi
                    ptx::mma_f16_ss(d1, ah, bl, IDESC, acc);     // D1 += hi*lo
                }
                ptx::mma_f16_ss(d1, al, bh, IDESC, 1u);          // D1 += lo*hi
                if constexpr (KIND == KIND_FP16X3) ptx::mma_f16_ss(d1, al, bl, IDESC, 1u);   // D1 += lo*lo
            }
        }
    }
}

// The MMA issuer's position in the stage ring.
struct MmaRing {
    uint32_t it;            // ring fills consumed so far
    int last_stage;         // stage of the last commit (-1: none yet)
    uint32_t last_parity;   // its phase parity
};

// All ring fills of one item (k-blocks g0 .. g1 - 1) for a block bj of NW
// columns: wait for the operands, issue the fill's MMAs, commit the stage
// back to the producer.  Returns false when a wait gave up.
template <int KIND, int NW, bool DIAG>
__device__ __forceinline__ bool mma_item(GramShared &sh, uint8_t *smem, uint32_t d0, int g0, int g1, MmaRing &r) {
    constexpr int UPK = KIND == KIND_TF32X3 ? 2 : 1;
    for (int u = g0 * UPK; u < g1 * UPK; ++u, ++r.it) {
        const int s = r.it % STAGES;
        if (!wait_or_abort(&sh.full[s], (r.it / STAGES) & 1, sh)) return false;
        ptx::tc_fence_after_sync();
        mma_fill<KIND, NW, DIAG>(d0, ptx::smem_u32(smem + s * STAGE_BYTES), u > g0 * UPK);
        ptx::mma_commit(ptx::smem_u32(&sh.empty[s]));
        r.last_stage = s;
        r.last_parity = (r.it / STAGES) & 1;
    }
    return true;
}

// Items of the narrow last column block: one instantiation per width (kept
// out of line, so that the issue loop of the full-width items stays small).
template <int KIND>
__device__ __noinline__ bool mma_item_narrow(int nw, bool diag, GramShared &sh, uint8_t *smem, uint32_t d0, int g0,
                                             int g1, MmaRing &r) {
#define CVX_NARROW(W)                                                                                     \
    case W:                                                                                               \
        return diag ? mma_item<KIND, W, true>(sh, smem, d0, g0, g1, r) : mma_item<KIND, W, false>(sh, smem, d0, g0, g1, r);
    switch (nw) {
        CVX_NARROW(16)
        CVX_NARROW(32)
        CVX_NARROW(48)
        CVX_NARROW(64)
        CVX_NARROW(80)
        CVX_NARROW(96)
        default:
            return diag ? mma_item<KIND, 112, true>(sh, smem, d0, g0, g1, r)
                        : mma_item<KIND, 112, false>(sh, smem, d0, g0, g1, r);
    }
#undef CVX_NARROW
}

template <int KIND, bool BATCHED>
__device__ __forceinline__ void gram_body(const PlanView &pl, const BatchTables &bt) {
    constexpr int UPK = KIND == KIND_TF32X3 ? 2 : 1;   // ring fills per k-block
    constexpr int TB = ops_tile_bytes(KIND);           // bytes of one operand tile
    extern __shared__ uint8_t smem_raw[];
    __shared__ GramShared sh;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const ItemSource<BATCHED> src(pl, bt);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(ptx::smem_u32(&sh.full[s]), 1);
            ptx::mbar_init(ptx::smem_u32(&sh.empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            ptx::mbar_init(ptx::smem_u32(&sh.acc_full[a]), 1);
            ptx::mbar_init(ptx::smem_u32(&sh.acc_empty[a]), 32 * EPI_WARPS);
        }
        sh.wait_ns = pl.wait_ns;
        sh.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == 1) {
        ptx::tmem_alloc(ptx::smem_u32(&sh.tmem_slot), TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before_sync();
    __syncthreads();
    ptx::tc_fence_after_sync();
    const uint32_t tmem = sh.tmem_slot;
    grid_dep_wait();
    grid_dep_launch();

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t idx = src.begin; idx < src.end && !sh.abort_flag; idx += src.step) {
                const ItemGeo ig = src(idx);
                const TileCoord tc = ig.tc;
                const bool diag = tc.bi == tc.bj;
                const int g0 = ig.g0, g1 = ig.g1;
                bool ok = true;
                // ring fills: one per k-block, or for TF32X3 one per 32-row half
                for (int u = g0 * UPK; u < g1 * UPK; ++u, ++it) {
                    const int g = u / UPK, h = u % UPK;
                    const int s = it % STAGES;
                    if (it >= STAGES && !wait_or_abort(&sh.empty[s], ((it / STAGES) - 1) & 1, sh)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = ptx::smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t bar = ptx::smem_u32(&sh.full[s]);
                    // B: the whole tile, or for a narrow last block the first nw
                    // columns of each of its two 16 KB parts (hi and lo, or the
                    // two TF32 row halves), nw * 128 bytes each
                    const uint32_t part = (uint32_t)ig.nw * 128u;
                    mbar_expect_tx(&sh.full[s], OPS_TILE_BYTES + (diag ? 0u : 2u * part));
                    bulk_copy(dst, ig.ops + ((int64_t)g * ig.nb + tc.bi) * TB + h * OPS_TILE_BYTES, OPS_TILE_BYTES,
                              bar);
                    if (!diag) {
                        const uint8_t *bsrc = ig.ops + ((int64_t)g * ig.nb + tc.bj) * TB + h * OPS_TILE_BYTES;
                        const uint32_t bdst = dst + OPS_TILE_BYTES;
                        if (ig.nw == TILE) {
                            bulk_copy(bdst, bsrc, OPS_TILE_BYTES, bar);
                        } else if constexpr (KIND == KIND_TF32) {
                            // keep the row halves 16 KB apart, as in a whole tile
                            bulk_copy(bdst, bsrc, part, bar);
                            bulk_copy(bdst + OP_BYTES, bsrc + OP_BYTES, part, bar);
                        } else {
                            // lo right after hi: [hi_B ; lo_B] is one operand of 2 nw rows
                            bulk_copy(bdst, bsrc, part, bar);
                            bulk_copy(bdst + part, bsrc + OP_BYTES, part, bar);
                        }
                    }
                }
                if (!ok) break;
            }
            // on an abort, copies already issued may still be landing in the ring
            drain_fills(sh.full, STAGES, it);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t n_done = 0;
            MmaRing ring{0u, -1, 0u};
            for (int64_t idx = src.begin; idx < src.end && !sh.abort_flag; idx += src.step) {
                const ItemGeo ig = src(idx);
                const bool diag = ig.tc.bi == ig.tc.bj;
                const int g0 = ig.g0, g1 = ig.g1;
                const int set = n_done & 1;
                // the epilogue must have drained this set (used two items ago)
                if (n_done >= 2 && !wait_or_abort(&sh.acc_empty[set], ((n_done / 2) - 1) & 1, sh)) break;
                ptx::tc_fence_after_sync();
                // B has nw columns (rows of the operand); D0 and D1 are nw TMEM
                // columns each, D1 right after D0
                const int nw = ig.nw;
                const uint32_t d0 = tmem + set * ACC_COLS;
                const bool ok = nw == TILE ? (diag ? mma_item<KIND, TILE, true>(sh, smem, d0, g0, g1, ring)
                                                   : mma_item<KIND, TILE, false>(sh, smem, d0, g0, g1, ring))
                                           : mma_item_narrow<KIND>(nw, diag, sh, smem, d0, g0, g1, ring);
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&sh.acc_full[set]));
                ++n_done;
            }
            // every MMA issued so far has completed once the last commit has
            // arrived; wait for it on every exit (another role may abort after
            // this thread's last check), so that no MMA still reads shared
            // memory or writes tensor memory when the CTA frees them
            if (ring.last_stage >= 0)
                ptx::mbar_wait_bounded(ptx::smem_u32(&sh.empty[ring.last_stage]), ring.last_parity, DRAIN_NS);
        }
    } else {
        // ------------------------------------------------------------- epilogue
        const int quad = warp & 3;   // TMEM lanes 32 quad .. 32 quad + 31
        const int row = quad * 32 + lane;
        uint32_t n_done = 0;
        for (int64_t idx = src.begin; idx < src.end && !sh.abort_flag; idx += src.step, ++n_done) {
            const ItemGeo ig = src(idx);
            const int set = n_done & 1;
            if (!wait_or_abort(&sh.acc_full[set], (n_done / 2) & 1, sh)) break;
            ptx::tc_fence_after_sync();
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + set * ACC_COLS;
            // FP16X3: D0 holds an integer below 2^24, stored exactly as int32,
            // and D1 as float.  BF16X3: D0 + D1 as float.  TF32: D1 alone.
            // Columns past nw of a narrow tile are not written (they stay zero).
            int32_t *out_hi = ig.out_hi;
            float *out_lo = ig.out_lo;
            const int nw = ig.nw;
#pragma unroll 1
            for (int col0 = 0; col0 < nw; col0 += 16) {
                uint32_t r0[16], r1[16];
                if constexpr (KIND != KIND_TF32) ptx::tmem_ld_32x32b_x16(base + col0, r0);
                ptx::tmem_ld_32x32b_x16(base + nw + col0, r1);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int64_t o = (int64_t)(col0 + q) * TILE + row;
                    if constexpr (KIND == KIND_FP16X3) {
                        out_hi[o] = __float2int_rn(__uint_as_float(r0[q]));
                        out_lo[o] = __uint_as_float(r1[q]);
                    } else if constexpr (KIND == KIND_BF16X3 || KIND == KIND_TF32X3) {
                        out_hi[o] = 0;
                        out_lo[o] = __uint_as_float(r0[q]) + __uint_as_float(r1[q]);
                    } else {
                        out_hi[o] = 0;
                        out_lo[o] = __uint_as_float(r1[q]);
                    }
                }
            }
            ptx::tc_fence_before_sync();
            mbar_arrive(&sh.acc_empty[set]);
        }
    }

    ptx::tc_fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        ptx::tc_fence_after_sync();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
    if (tid == 0 && sh.abort_flag) atomicOr(BATCHED ? bt.views[0].err : pl.err, DEV_ERR_TIMEOUT);
}

template <int KIND>
__global__ void __launch_bounds__(THREADS, 1) k_gram_tc(const __grid_constant__ PlanView pl) {
    BatchTables none = {};
    gram_body<KIND, false>(pl, none);
}

// Batched: CTA b walks its own list of (problem, item) pairs.
template <int KIND>
__global__ void __launch_bounds__(THREADS, 1) k_gram_tc_batched(const __grid_constant__ BatchTables bt) {
    gram_body<KIND, true>(bt.views[0], bt);
}

}  // namespace

cudaError_t convert_split(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                          cudaStream_t st) {
    const int x_vec = ((uintptr_t)X % 16 == 0) && (ldx % 4 == 0);
    const int mp = pl->ypack_width;
    const int ybw = mp;   // a multiple of 4
    const bool rows_ok = pl->in_dtype == CV_F32 && x_vec && pl->v.K % 4 == 0 && pl->ypack != nullptr;
    // Gathered rows: whole-row fills (measured on N = 1e6, K = 1024, M = 16,
    // random folds, against the bulk converter's 512-byte row pieces: FP16X3
    // 1.41 against 2.37 ms, BF16X3 1.39 against 2.39, TF32X3 2.03 against
    // 2.70, TF32 1.24 against 2.35).
    if (rows_ok && pl->gathered && pl->v.D <= CR_CONV * CR_MAX_COLS) {
        // whole rows per ring fill: 16 rows while three stages fit, else 8
        RowGeom geo;
        geo.mp = mp;
        geo.stages = 0;
        for (int R = 16; R >= 8 && geo.stages < 3; R /= 2) {
            geo.rows = R;
            geo.xbytes = R * pl->v.K * 4;
            geo.stage_bytes = (geo.xbytes + R * mp * 4 + 1023) / 1024 * 1024;
            geo.stages = std::min(CB_MAX_STAGES, (216 * 1024) / geo.stage_bytes);
        }
        if (geo.stages >= 3) {
            const int smem = geo.stages * geo.stage_bytes + 1024;
            const int k = pl->v.kind;
            auto kern = geo.rows == 16 ? (k == KIND_FP16X3   ? k_convert_rows<KIND_FP16X3, 16>
                                          : k == KIND_BF16X3 ? k_convert_rows<KIND_BF16X3, 16>
                                          : k == KIND_TF32X3 ? k_convert_rows<KIND_TF32X3, 16>
                                                             : k_convert_rows<KIND_TF32, 16>)
                                       : (k == KIND_FP16X3   ? k_convert_rows<KIND_FP16X3, 8>
                                          : k == KIND_BF16X3 ? k_convert_rows<KIND_BF16X3, 8>
                                          : k == KIND_TF32X3 ? k_convert_rows<KIND_TF32X3, 8>
                                                             : k_convert_rows<KIND_TF32, 8>);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            const int grid = (int)std::min<int64_t>(pl->v.nkb, pl->num_sms);
            ++pl->launches;
            return launch_pdl(kern, dim3(grid), dim3(CR_THREADS), (size_t)smem, st, pl->v, (const float *)X, ldx,
                              (const float *)pl->ypack, geo);
        }
    }
    if (rows_ok && ybw <= 64 && tensor_map_encoder() != nullptr) {
        // Yp (Y and the ones column in 16-byte rows) was packed by the shift
        // estimate's kernel, which runs first on the stream
        const int64_t n = pl->v.N;
        CUtensorMap tm_x, tm_y;
        if (!make_map_f32(&tm_x, X, pl->v.K, n, ldx, TILE, KB) || !make_map_f32(&tm_y, pl->ypack, mp, n, mp, ybw, KB))
            return cudaErrorInvalidValue;
        ConvGeom geo;
        geo.mp = mp;
        geo.ybw = ybw;
        geo.stage_bytes = (CB_XBYTES + KB * ybw * 4 + 1023) / 1024 * 1024;
        geo.stages = std::min(CB_MAX_STAGES, (220 * 1024) / geo.stage_bytes);
        const int smem = geo.stages * geo.stage_bytes + 1024;
        auto kern = pl->v.kind == KIND_FP16X3   ? k_convert_bulk<KIND_FP16X3>
                    : pl->v.kind == KIND_BF16X3 ? k_convert_bulk<KIND_BF16X3>
                    : pl->v.kind == KIND_TF32X3 ? k_convert_bulk<KIND_TF32X3>
                                                : k_convert_bulk<KIND_TF32>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        const int grid = (int)std::min<int64_t>(pl->v.nkb, pl->num_sms);
        ++pl->launches;
        return launch_pdl(kern, dim3(grid), dim3(CB_THREADS), (size_t)smem, st, pl->v, (const float *)X, ldx,
                          (const float *)pl->ypack, geo, tm_x, tm_y);
    }
    ++pl->launches;
    const int kind = pl->v.kind;
    if (pl->in_dtype == CV_F32) {
        // whole rows read with plain loads (measured on N = 4e5, K = 1021,
        // M = 16: FP16X3 conversion 0.95 ms with 128-column cp.async pieces)
        auto kern = kind == KIND_FP16X3 ? k_convert_direct<KIND_FP16X3>
                    : kind == KIND_BF16X3 ? k_convert_direct<KIND_BF16X3>
                    : kind == KIND_TF32X3 ? k_convert_direct<KIND_TF32X3>
                                          : k_convert_direct<KIND_TF32>;
        // runs short enough that every SM gets two blocks or more
        const int run = (int)std::max<int64_t>(
            1, std::min<int64_t>(direct_run(pl->v.D), pl->v.nkb / (2 * (int64_t)pl->num_sms)));
        return launch_pdl(kern, dim3((unsigned)((pl->v.nkb + run - 1) / run)), dim3(CD_THREADS), 0, st, pl->v,
                          (const float *)X, ldx, (const float *)Y, ldy, run);
    }
    const int per_cb = (int)std::min<int64_t>(pl->v.nkb, (int64_t)8 * pl->num_sms);
    dim3 grid(per_cb, pl->v.nb);
    auto kern = kind == KIND_FP16X3 ? k_convert<double, KIND_FP16X3>
                : kind == KIND_BF16X3 ? k_convert<double, KIND_BF16X3>
                : kind == KIND_TF32X3 ? k_convert<double, KIND_TF32X3>
                                      : k_convert<double, KIND_TF32>;
    return launch_pdl(kern, grid, dim3(256), 0, st, pl->v, (const double *)X, ldx, (const double *)Y, ldy, 0);
}

cudaError_t gram_tc(const cv_plan_s *pl, cudaStream_t st) {
    const int64_t items = (int64_t)pl->v.nsegs * pl->v.ntiles;
    const int grid = (int)(items < pl->num_sms ? items : pl->num_sms);
    auto kern = pl->v.kind == KIND_FP16X3   ? k_gram_tc<KIND_FP16X3>
                : pl->v.kind == KIND_BF16X3 ? k_gram_tc<KIND_BF16X3>
                : pl->v.kind == KIND_TF32X3 ? k_gram_tc<KIND_TF32X3>
                                            : k_gram_tc<KIND_TF32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    ++pl->launches;
    return launch_pdl(kern, dim3(grid), dim3(THREADS), (size_t)SMEM_BYTES, st, pl->v);
}

cudaError_t convert_batched(const BatchTables &bt, const BatchArgs &ba, cudaStream_t st) {
    auto kern = bt.kind == KIND_FP16X3 ? k_convert_batched<KIND_FP16X3>
                : bt.kind == KIND_BF16X3 ? k_convert_batched<KIND_BF16X3>
                : bt.kind == KIND_TF32X3 ? k_convert_batched<KIND_TF32X3>
                                         : k_convert_batched<KIND_TF32>;
    return launch_pdl(kern, dim3(bt.n_conv), dim3(CD_THREADS), 0, st, bt, ba);
}

cudaError_t gram_tc_batched(const BatchTables &bt, cudaStream_t st) {
    auto kern = bt.kind == KIND_FP16X3 ? k_gram_tc_batched<KIND_FP16X3>
                : bt.kind == KIND_BF16X3 ? k_gram_tc_batched<KIND_BF16X3>
                : bt.kind == KIND_TF32X3 ? k_gram_tc_batched<KIND_TF32X3>
                                         : k_gram_tc_batched<KIND_TF32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    return launch_pdl(kern, dim3(bt.gram_ctas), dim3(THREADS), (size_t)SMEM_BYTES, st, bt);
}

}  // namespace cvx
