// gram_tc.cu -- tcgen05 tensor-core contraction of the fold-grouped Gram in
// split FP16 precision (CV_PREC_FP16X3).
//
// Each (segment, tile) work item forms the 128 x 128 tile (bi, bj) of
// H_S = W_S^T W_S over the segment's rows S (one fold), W = [X' | Y' | 1] with
// v = (x - s_c) * 2^e_c (the shift and power-of-two scale from the shift
// estimate).  That is Algorithm 7 steps 8, 17 and 19 for the rows of S in one
// contraction (the sums and sums of squares sit in the ones column and on the
// diagonal).
//
// Precision.  Every v is split into an integer part hi = rint(v), exact in
// FP16 while |hi| <= 2048, and a remainder lo = fp16(v - hi), |lo| <= 1/2, so
// v = hi + lo to within 2^-13 (FP16 keeps 11 bits of the remainder).  The
// scale maps the sampled column maximum to 2^B, with B chosen by the plan from
// the longest segment so that sums of hi * hi over a segment stay below 2^24.
// The tile is accumulated by tcgen05.mma (kind::f16) into two FP32
// tensor-memory accumulators:
//   D0 = sum hi * hi                 integer partial sums below 2^24: exact,
//                                    whatever rounding the accumulator uses;
//   D1 = sum hi * lo + lo * hi + lo * lo
//                                    about 2^-B of D0, so its own rounding is
//                                    far below the 1e-6 target.
// The item writes D0 + D1 as an FP64 partial tile; every reduction after that
// is FP64.
//
// Pipeline.  A persistent CTA (one per SM) walks the work items
// b, b + gridDim.x, ... with
//   converter groups   8 warps each (2 groups for FP32 inputs, 1 for FP64);
//                      group g takes every k-block (64 rows) with global index
//                      it % groups == g, gathers its rows through the
//                      fold-sorted order, shifts, scales, splits and stores
//                      hi / lo into a K-major 128-byte-swizzled operand stage,
//                      then arrives on the stage's `full` mbarrier.  While one
//                      group waits on its loads, the other converts;
//   MMA warp           one thread waits on `full`, issues 16 MMAs
//                      (M = N = 128, K = 16) per k-block and commits them to
//                      the stage's `empty` mbarrier; after an item's last
//                      k-block it commits to `acc_full`;
//   epilogue           converter group 0 reads D0 and D1 from tensor memory
//                      (two warps per 32-lane quadrant, 64 columns each),
//                      stores the FP64 partial tile and arrives on
//                      `acc_empty`, which the next item's MMAs wait for.
// Three operand stages of 64 KB each.  Every mbarrier wait is bounded: on
// expiry the waiting thread raises a CTA-wide abort flag, every role leaves
// its loop, the MMA thread drains its last commit (bounded), the tensor
// memory is freed and DEV_ERR_TIMEOUT is recorded.
#include <cuda_fp16.h>

#include "cvx_internal.cuh"
#include "tc_ptx.cuh"

namespace cvx {
namespace {

constexpr int KB = 64;                         // rows per k-block: one 128-byte swizzle row of FP16
constexpr int OP_BYTES = TILE * KB * 2;        // one FP16 operand tile: 16 KB
constexpr int TC_STAGES = 3;
constexpr int TC_STAGE_BYTES = 4 * OP_BYTES;   // A_hi, A_lo, B_hi, B_lo
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024;
constexpr int GROUP_THREADS = 256;
constexpr int ROWS_PER_THREAD = 32;
constexpr uint32_t TMEM_COLS = 256;            // D0 at column 0, D1 at column 128
constexpr uint64_t WAIT_TIMEOUT_NS = 1000000000ull;   // 1 s
constexpr float FP16_OVERFLOW = 65520.0f;            // smallest float that rounds to inf

template <typename T>
struct Cfg {
    static constexpr int GROUPS = sizeof(T) == 4 ? 2 : 1;
    static constexpr int THREADS = GROUPS * GROUP_THREADS + 32;
    // Registers per thread for the one resident CTA: warps are spread over
    // the SM's four 16K-register partitions, so the busiest partition holds
    // ceil(warps / 4) warps; the count is rounded down to a multiple of 8.
    static constexpr int WARPS_PER_PART = (THREADS / 32 + 3) / 4;
    static constexpr int REG_LIMIT = ((16384 / (WARPS_PER_PART * 32)) / 8) * 8;
    static constexpr int MAX_REGS = REG_LIMIT > 255 ? 248 : REG_LIMIT;
};

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
    cs.ptr = nullptr;
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

// Split two consecutive-row values into integer hi and remainder lo FP16
// pairs: hi = fp16(rint(v)), lo = fp16(v - hi).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &lo, bool &bad) {
    const __half2 h = __floats2half2_rn(rintf(a), rintf(b));
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = h2_bits(h);
    lo = h2_bits(l);
    bad |= (fabsf(a) >= FP16_OVERFLOW) | (fabsf(b) >= FP16_OVERFLOW);
}

__device__ __forceinline__ void split_pair(double a, double b, uint32_t &hi, uint32_t &lo, bool &bad) {
    const __half ha = __double2half(rint(a)), hb = __double2half(rint(b));
    const __half la = __double2half(a - (double)__half2float(ha));
    const __half lb = __double2half(b - (double)__half2float(hb));
    hi = h2_bits(__halves2half2(ha, hb));
    lo = h2_bits(__halves2half2(la, lb));
    bad |= (fabs(a) >= (double)FP16_OVERFLOW) | (fabs(b) >= (double)FP16_OVERFLOW);
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

// Load the thread's 32 rows of its column; row k's index comes from lane k.
template <typename T>
__device__ __forceinline__ void load_rows(const ColSrc<T> &cs, int32_t my_row, T (&x)[ROWS_PER_THREAD]) {
#pragma unroll
    for (int k = 0; k < ROWS_PER_THREAD; ++k) {
        const int32_t n = __shfl_sync(0xffffffffu, my_row, k);
        x[k] = (cs.kind == COL_DATA && n >= 0) ? __ldg(cs.ptr + (int64_t)n * cs.ld) : T(0);
    }
}

// Convert the thread's 32 rows and store them as four 16-byte chunks of its
// tile row in the K-major SW128 layout:
// byte offset of (row c, k) = c * 128 + ((k / 8) ^ (c % 8)) * 16 + (k % 8) * 2.
// Rows past the segment's end (row index -1) are stored as zero.
template <typename T>
__device__ __forceinline__ void convert_rows(const ColSrc<T> &cs, int32_t my_row, const T (&x)[ROWS_PER_THREAD],
                                             uint8_t *hi_tile, uint8_t *lo_tile, int c, int h, bool &bad) {
    using V = typename Acc<T>::type;
    const unsigned valid = __ballot_sync(0xffffffffu, my_row >= 0);
    const V fill = cs.kind == COL_ONES ? V(1) : V(0);
#pragma unroll
    for (int g = 0; g < ROWS_PER_THREAD / 8; ++g) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k0 = 8 * g + 2 * q;
            V a = cs.kind == COL_DATA ? prep_value<T>(cs, x[k0]) : fill;
            V b = cs.kind == COL_DATA ? prep_value<T>(cs, x[k0 + 1]) : fill;
            if (!((valid >> k0) & 1u)) a = V(0);
            if (!((valid >> (k0 + 1)) & 1u)) b = V(0);
            split_pair(a, b, hw[q], lw[q], bad);
        }
        const int chunk = 4 * h + g;
        const uint32_t off = (uint32_t)c * 128u + ((uint32_t)(chunk ^ (c & 7)) << 4);
        *reinterpret_cast<uint4 *>(hi_tile + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(lo_tile + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

struct TcShared {
    uint64_t full[TC_STAGES];    // converters -> MMA: stage written (count = GROUP_THREADS)
    uint64_t empty[TC_STAGES];   // MMA -> converters: stage consumed (tcgen05.commit)
    uint64_t acc_full;           // MMA -> epilogue: accumulators final (tcgen05.commit)
    uint64_t acc_empty;          // epilogue -> MMA: accumulators drained (count = GROUP_THREADS)
    uint32_t tmem_slot;
    volatile int abort_flag;
};

// Bounded wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, TcShared &sh) {
    const uint32_t a = ptx::smem_u32(bar);
    if (ptx::mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (true) {
        if (ptx::mbar_try_wait(a, parity)) return true;
        if (sh.abort_flag) return false;
        if (ptx::globaltimer_ns() - t0 > WAIT_TIMEOUT_NS) {
            sh.abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}

template <typename T>
__global__ void __maxnreg__(Cfg<T>::MAX_REGS)
    k_gram_tc(PlanView pl, const T *__restrict__ X, int64_t ldx, const T *__restrict__ Y, int64_t ldy) {
    constexpr int GROUPS = Cfg<T>::GROUPS;
    constexpr int CONV_THREADS = GROUPS * GROUP_THREADS;
    constexpr int MMA_WARP = CONV_THREADS / 32;
    extern __shared__ uint8_t smem_raw[];
    __shared__ TcShared sh;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_items = (int64_t)pl.nsegs * pl.ntiles;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            ptx::mbar_init(ptx::smem_u32(&sh.full[s]), GROUP_THREADS);
            ptx::mbar_init(ptx::smem_u32(&sh.empty[s]), 1);
        }
        ptx::mbar_init(ptx::smem_u32(&sh.acc_full), 1);
        ptx::mbar_init(ptx::smem_u32(&sh.acc_empty), GROUP_THREADS);
        sh.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    if (warp == MMA_WARP) {
        ptx::tmem_alloc(ptx::smem_u32(&sh.tmem_slot), TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before_sync();
    __syncthreads();
    ptx::tc_fence_after_sync();
    const uint32_t tmem = sh.tmem_slot;
    bool bad = false;

    if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = ptx::idesc_f16_f32(TILE, TILE);
            uint32_t it = 0, n_done = 0;
            int last_stage = -1;
            uint32_t last_parity = 0;
            for (int64_t item = blockIdx.x; item < n_items && !sh.abort_flag; item += gridDim.x) {
                const Segment sg = pl.segs[item / pl.ntiles];
                const TileCoord tc = pl.tiles[item % pl.ntiles];
                const bool diag = tc.bi == tc.bj;
                const int nkb = (sg.end - sg.begin + KB - 1) / KB;
                // the previous item's epilogue must have drained the accumulators
                if (n_done > 0 && !wait_or_abort(&sh.acc_empty, (n_done - 1) & 1, sh)) break;
                ptx::tc_fence_after_sync();
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % TC_STAGES;
                    if (!wait_or_abort(&sh.full[s], (it / TC_STAGES) & 1, sh)) {
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after_sync();
                    const uint32_t a_hi = ptx::smem_u32(smem + s * TC_STAGE_BYTES), a_lo = a_hi + OP_BYTES;
                    const uint32_t b_hi = diag ? a_hi : a_hi + 2 * OP_BYTES;
                    const uint32_t b_lo = diag ? a_lo : a_hi + 3 * OP_BYTES;
                    const uint32_t d0 = tmem, d1 = tmem + TILE;
#pragma unroll
                    for (int kk = 0; kk < KB / 16; ++kk) {
                        const uint32_t o = kk * 32;   // 16 FP16 along K = 32 bytes
                        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                        const uint64_t ah = ptx::desc_kmajor_sw128(a_hi + o), al = ptx::desc_kmajor_sw128(a_lo + o);
                        const uint64_t bh = ptx::desc_kmajor_sw128(b_hi + o), bl = ptx::desc_kmajor_sw128(b_lo + o);
                        ptx::mma_f16_ss(d0, ah, bh, IDESC, acc);
                        ptx::mma_f16_ss(d1, ah, bl, IDESC, acc);
                        ptx::mma_f16_ss(d1, al, bh, IDESC, 1u);
                        ptx::mma_f16_ss(d1, al, bl, IDESC, 1u);
                    }
                    ptx::mma_commit(ptx::smem_u32(&sh.empty[s]));
                    last_stage = s;
                    last_parity = (it / TC_STAGES) & 1;
                }
                if (!ok) break;
                ptx::mma_commit(ptx::smem_u32(&sh.acc_full));
                ++n_done;
            }
            if (sh.abort_flag && last_stage >= 0) {
                // drain the MMAs still in flight (bounded) before the columns are freed
                ptx::mbar_wait_bounded(ptx::smem_u32(&sh.empty[last_stage]), last_parity, WAIT_TIMEOUT_NS);
            }
        }
    } else {
        // ------------------------------------------------------ converters
        const int group = tid / GROUP_THREADS;
        const int t = tid % GROUP_THREADS;
        const int c = t % TILE, h = t / TILE;
        uint32_t it = 0, n_done = 0;
        for (int64_t item = blockIdx.x; item < n_items && !sh.abort_flag; item += gridDim.x) {
            const Segment sg = pl.segs[item / pl.ntiles];
            const TileCoord tc = pl.tiles[item % pl.ntiles];
            const bool diag = tc.bi == tc.bj;
            const int nkb = (sg.end - sg.begin + KB - 1) / KB;
            const ColSrc<T> src_a = column_source(pl, X, ldx, Y, ldy, tc.bi * TILE + c);
            const ColSrc<T> src_b = column_source(pl, X, ldx, Y, ldy, tc.bj * TILE + c);
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb, ++it) {
                if ((int)(it % GROUPS) != group) continue;
                const int s = it % TC_STAGES;
                // lane l holds the row index of row 32 h + l of this k-block
                const int r = sg.begin + kb * KB + ROWS_PER_THREAD * h + lane;
                const int32_t my_row = r < sg.end ? pl.perm[r] : -1;
                T x[ROWS_PER_THREAD];
                load_rows<T>(src_a, my_row, x);
                if (it >= TC_STAGES && !wait_or_abort(&sh.empty[s], ((it / TC_STAGES) - 1) & 1, sh)) {
                    ok = false;
                    break;
                }
                uint8_t *stage = smem + s * TC_STAGE_BYTES;
                convert_rows<T>(src_a, my_row, x, stage, stage + OP_BYTES, c, h, bad);
                if (!diag) {
                    load_rows<T>(src_b, my_row, x);
                    convert_rows<T>(src_b, my_row, x, stage + 2 * OP_BYTES, stage + 3 * OP_BYTES, c, h, bad);
                }
                ptx::fence_proxy_async_smem();
                mbar_arrive(&sh.full[s]);
            }
            if (!ok) break;
            // -------------------------------------------------- epilogue (group 0)
            if (group == 0) {
                if (!wait_or_abort(&sh.acc_full, n_done & 1, sh)) break;
                ptx::tc_fence_after_sync();
                const int w = t >> 5;                    // 0..7
                const int quad = w & 3, half = w >> 2;  // TMEM lanes 32 quad .., columns 64 half ..
                const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
                double *out = pl.partials + item * TILE_ELEMS;
                const int row = quad * 32 + lane;
#pragma unroll 1
                for (int chunk = 0; chunk < 2; ++chunk) {
                    const int col0 = half * 64 + chunk * 32;
                    uint32_t r0[32], r1[32];
                    ptx::tmem_ld_32x32b_x32(lane_base + col0, r0);
                    ptx::tmem_ld_32x32b_x32(lane_base + TILE + col0, r1);
                    ptx::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        out[(int64_t)(col0 + q) * TILE + row] =
                            (double)__uint_as_float(r0[q]) + (double)__uint_as_float(r1[q]);
                }
                ptx::tc_fence_before_sync();
                mbar_arrive(&sh.acc_empty);
            }
            ++n_done;
        }
    }

    ptx::tc_fence_before_sync();
    __syncthreads();
    if (warp == MMA_WARP) {
        ptx::tc_fence_after_sync();
        ptx::tmem_dealloc(tmem, TMEM_COLS);
    }
    if (tid == 0 && sh.abort_flag) atomicOr(pl.err, DEV_ERR_TIMEOUT);
    if (bad) atomicOr(pl.err, DEV_ERR_RANGE);
}

}  // namespace

cudaError_t gram_tc(const cv_plan_s *pl, const void *X, int64_t ldx, const void *Y, int64_t ldy,
                    cudaStream_t st) {
    const int64_t items = (int64_t)pl->v.nsegs * pl->v.ntiles;
    const int grid = (int)(items < pl->num_sms ? items : pl->num_sms);
    cudaError_t e;
    if (pl->in_dtype == CV_F32) {
        e = cudaFuncSetAttribute(k_gram_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        k_gram_tc<float><<<grid, Cfg<float>::THREADS, TC_SMEM_BYTES, st>>>(pl->v, (const float *)X, ldx,
                                                                          (const float *)Y, ldy);
    } else {
        e = cudaFuncSetAttribute(k_gram_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        k_gram_tc<double><<<grid, Cfg<double>::THREADS, TC_SMEM_BYTES, st>>>(pl->v, (const double *)X, ldx,
                                                                            (const double *)Y, ldy);
    }
    return cudaGetLastError();
}

}  // namespace cvx
