// fold_sort.cu -- Algorithm 1 (Section 3) on the device: validate the fold ids,
// count the rows of every fold, and list the rows of each fold in increasing
// row order (a stable counting sort of the row indices by fold id).
//
// The sort is a least-significant-digit radix sort on 8-bit digits of the
// fold id, so ceil(log2(P) / 8) passes; each pass is stable, which keeps the
// rows of a fold in their original order and makes the whole library's
// summation order deterministic.
#include <algorithm>

#include "cvx_internal.cuh"

namespace cvx {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // rows per block
static_assert(RS_TILE == FOLD_SORT_ROWS_PER_BLOCK, "the scratch size formula assumes this tile");
constexpr int SMEM_HIST_MAX = 8192;              // folds counted in shared memory

__global__ void k_fold_count(const int32_t *__restrict__ folds, int64_t N, int32_t P,
                             unsigned long long *__restrict__ counts, int *__restrict__ bad) {
    extern __shared__ unsigned int sh[];
    const bool use_smem = P <= SMEM_HIST_MAX;
    if (use_smem) {
        for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    int local_bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = folds[i];
        if (f < 0 || f >= P) {
            local_bad = 1;
        } else if (use_smem) {
            atomicAdd(&sh[f], 1u);
        } else {
            atomicAdd(&counts[f], 1ull);
        }
    }
    if (local_bad) atomicOr(bad, 1);
    if (use_smem) {
        __syncthreads();
        for (int i = threadIdx.x; i < P; i += blockDim.x)
            if (sh[i]) atomicAdd(&counts[i], (unsigned long long)sh[i]);
    }
}

__global__ void k_radix_hist(const int32_t *__restrict__ keys, int64_t N, int shift, int nblk,
                             unsigned int *__restrict__ blockhist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        const int64_t r = base + i;
        if (r < N) atomicAdd(&h[(keys[r] >> shift) & 255], 1u);
    }
    __syncthreads();
    blockhist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// In-place exclusive scan of n unsigned ints with one block of 1024 threads.
__global__ void k_scan_exclusive(unsigned int *__restrict__ data, int64_t n) {
    __shared__ unsigned int warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t lo = tid * per, hi = min(n, lo + per);
    unsigned int local = 0;
    for (int64_t i = lo; i < hi; ++i) local += data[i];
    unsigned int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned int w = warp_sums[lane];
        unsigned int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        warp_sums[lane] = wi - w;   // exclusive prefix of warp totals
    }
    __syncthreads();
    unsigned int run = warp_sums[warp] + incl - local;
    for (int64_t i = lo; i < hi; ++i) {
        const unsigned int v = data[i];
        data[i] = run;
        run += v;
    }
}

// Stable scatter of one radix pass.  Within a block the 4096 rows are taken
// in 16 sub-tiles of 256, in order; inside a sub-tile a row's rank among rows
// of the same digit is (rows of that digit in earlier warps) + (earlier lanes
// of its own warp with that digit).
__global__ void k_radix_scatter(const int32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                int32_t *__restrict__ kout, int32_t *__restrict__ vout, int64_t N,
                                int shift, int nblk, const unsigned int *__restrict__ scanned) {
    __shared__ unsigned int base[256];
    __shared__ unsigned int wcount[RS_THREADS / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = scanned[(int64_t)tid * nblk + blockIdx.x];
    const unsigned int lt_mask = (1u << lane) - 1u;
    for (int sub = 0; sub < RS_ITEMS; ++sub) {
        for (int w = 0; w < RS_THREADS / 32; ++w) wcount[w][tid] = 0;
        __syncthreads();
        const int64_t i = (int64_t)blockIdx.x * RS_TILE + (int64_t)sub * RS_THREADS + tid;
        const bool valid = i < N;
        const int32_t key = valid ? kin[i] : 0;
        const int digit = valid ? ((key >> shift) & 255) : 256;
        const unsigned int peers = __match_any_sync(0xffffffffu, digit);
        const unsigned int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcount[warp][digit] = __popc(peers);
        __syncthreads();
        unsigned int run = 0;
        unsigned int my_off = 0;
        // thread `tid` owns digit `tid`: prefix over warps
        unsigned int offs_w[RS_THREADS / 32];
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) {
            offs_w[w] = run;
            run += wcount[w][tid];
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < RS_THREADS / 32; ++w) wcount[w][tid] = offs_w[w];
        __syncthreads();
        if (valid) {
            my_off = base[digit] + wcount[warp][digit] + rank;
            kout[my_off] = key;
            vout[my_off] = vin ? vin[i] : (int32_t)i;
        }
        __syncthreads();
        base[tid] += run;
        __syncthreads();
    }
}

}  // namespace

cudaError_t fold_count(const int32_t *folds, int64_t N, int32_t P, unsigned long long *counts,
                       int *bad, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (N + threads * 8 - 1) / (threads * 8);
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    const size_t smem = P <= SMEM_HIST_MAX ? sizeof(unsigned int) * (size_t)P : 0;
    k_fold_count<<<(unsigned)blocks, threads, smem, st>>>(folds, N, P, counts, bad);
    return cudaGetLastError();
}

size_t fold_sort_tmp_bytes(int64_t N) { return fold_sort_tmp_bytes_for(N); }

namespace {

// Number of places where the fold-sorted order leaves a run of consecutive
// rows: n with perm[n + 1] != perm[n] + 1.
__global__ void k_perm_breaks(const int32_t *__restrict__ perm, int64_t N, unsigned long long *__restrict__ breaks) {
    unsigned long long local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + 1 < N; i += (int64_t)gridDim.x * blockDim.x)
        local += perm[i + 1] != perm[i] + 1;
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(breaks, local);
}

}  // namespace

cudaError_t perm_breaks(const int32_t *perm, int64_t N, unsigned long long *breaks, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>(1024, (N + 255) / 256);
    k_perm_breaks<<<(unsigned)std::max<int64_t>(1, blocks), 256, 0, st>>>(perm, N, breaks);
    return cudaGetLastError();
}

cudaError_t fold_sort(const int32_t *folds, int64_t N, int32_t P, int32_t *perm, void *tmp,
                      size_t tmp_bytes, cudaStream_t st) {
    if (tmp_bytes < fold_sort_tmp_bytes(N)) return cudaErrorInvalidValue;
    const int nblk = (int)((N + RS_TILE - 1) / RS_TILE);
    int32_t *ka = (int32_t *)tmp;
    int32_t *kb = ka + N;
    int32_t *va = kb + N;
    int32_t *vb = va + N;
    unsigned int *hist = (unsigned int *)(vb + N);
    int bits = 0;
    while (bits < 31 && (1ll << bits) < (int64_t)P) ++bits;
    const int passes = bits == 0 ? 1 : (bits + 7) / 8;
    const int32_t *kin = folds;
    const int32_t *vin = nullptr;   // identity on the first pass
    for (int ps = 0; ps < passes; ++ps) {
        const bool last = ps == passes - 1;
        int32_t *kout = (ps % 2 == 0) ? ka : kb;
        int32_t *vout = last ? perm : ((ps % 2 == 0) ? va : vb);
        k_radix_hist<<<nblk, RS_THREADS, 0, st>>>(kin, N, 8 * ps, nblk, hist);
        k_scan_exclusive<<<1, 1024, 0, st>>>(hist, (int64_t)nblk * 256);
        k_radix_scatter<<<nblk, RS_THREADS, 0, st>>>(kin, vin, kout, vout, N, 8 * ps, nblk, hist);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        kin = kout;
        vin = vout;
    }
    return cudaSuccess;
}

}  // namespace cvx
