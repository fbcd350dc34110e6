// Connected density correlator of Eqs. 5 and 10 as a Gram contraction on
// the tcgen05 tensor cores, in BF16x3 split precision.
//
//   C_t = (1/M) (X_t - mu_t)^T (X_t - mu_t),   X_t: M samples x K = 2N sites
//
// The centred data y = x - mu are split as y = hi + lo with hi = bf16_rn(y),
// lo = bf16_rn(y - hi); the product y_k y_l is approximated by
// hi_k hi_l + hi_k lo_l + lo_k hi_l (the lo*lo term, ~2^-16 relative, is
// dropped), each a bf16 MMA with FP32 accumulation in tensor memory.
//
// Two kernels per batch of output times:
//  1. split_kernel centres, splits and transposes X_t into two bf16 arrays
//     hi, lo of shape [t][Kd][Mp] (sites x samples, samples contiguous;
//     Kd = max(K, 128) rows, Mp = M rounded up to 64 samples, zero padded);
//  2. gram_tc_kernel, one CTA per (time, 128 x 128 tile of the upper
//     triangle), warp-specialised: warp 0 streams 64-sample chunks of the
//     operands with TMA (128-byte swizzle, three stages), warp 1 issues the
//     MMAs (M = N = 128, K = 16 per instruction) into one of two tensor-memory
//     accumulators, and eight epilogue warps drain each 1024-sample segment
//     of the FP32 accumulator into FP32 register sums while the next segment
//     accumulates.  Segments bound the length of every FP32 tensor-core sum
//     (the variances are long same-sign sums) to 1024 terms; the sum over
//     segments adds one rounding per segment (64 at M = 65536), less than
//     the rounding inside one segment.  The epilogue writes conn (both triangles) and g2 directly.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ftwa_internal.h"
#include "ptx.cuh"

namespace ftwa {

namespace gram {

constexpr int kTile = 128;                   // output tile edge (sites)
constexpr int kChunk = 64;                   // samples per operand image (128 bytes of bf16)
constexpr int kImage = kTile * kChunk * 2;   // 16 KB per operand image
constexpr int kStages = 3;
constexpr int kSegChunks = 16;               // chunks per FP32 accumulation segment (1024 samples)
constexpr int kEpiWarps = 8;
constexpr int kThreadsG = 32 * (2 + kEpiWarps);

// ---- 1. centre, split, transpose ------------------------------------------------
// tile: 64 samples x 128 sites.  Lane l reads sites l, l + 32, l + 64, l + 96
// of a sample row (coalesced 128-byte rows), the centred values are
// transposed through shared memory (odd row pitch: conflict-free writes), and
// each thread splits 8 consecutive samples of one site into 16 bytes of hi
// and 16 bytes of lo (8 lanes write one 128-byte row segment).
constexpr int kSplitSites = 128;

__global__ void __launch_bounds__(256) split_kernel(const float *X, const double *mu, __nv_bfloat16 *hi,
                                                   __nv_bfloat16 *lo, long long M, int K, int Kd, long long Mp,
                                                   int t0)
{
    __shared__ float tile[kSplitSites][kChunk + 1];
    const long long m0 = (long long)blockIdx.x * kChunk;
    const int k0 = blockIdx.y * kSplitSites;
    const int tl = blockIdx.z, t = t0 + tl;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float *Xt = X + (long long)t * M * K;
    float mr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = k0 + lane + 32 * i;
        mr[i] = k < K ? (float)mu[(long long)t * K + k] : 0.0f;
    }
    float v[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long m = m0 + w + 8 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + lane + 32 * i;
            v[j][i] = (m < M && k < K) ? Xt[m * K + k] : 0.0f;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long m = m0 + w + 8 * j;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + lane + 32 * i;
            tile[lane + 32 * i][w + 8 * j] = (m < M && k < K) ? v[j][i] - mr[i] : 0.0f;
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int id = threadIdx.x + 256 * u;
        const int sl = id >> 3, o = id & 7;        // site of the tile, sample octet
        const int k = k0 + sl;
        if (k >= Kd) continue;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float y0 = tile[sl][8 * o + 2 * j], y1 = tile[sl][8 * o + 2 * j + 1];
            const __nv_bfloat162 hb = __floats2bfloat162_rn(y0, y1);
            const float2 hf = __bfloat1622float2(hb);
            const __nv_bfloat162 lb = __floats2bfloat162_rn(y0 - hf.x, y1 - hf.y);
            hw[j] = *reinterpret_cast<const uint32_t *>(&hb);
            lw[j] = *reinterpret_cast<const uint32_t *>(&lb);
        }
        const long long off = ((long long)tl * Kd + k) * Mp + m0 + 8 * o;
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(lo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// ---- 2. the contraction ------------------------------------------------------------
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout a 128-byte-swizzled TMA box of 64 bf16 x 128
// rows leaves in shared memory)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// instruction descriptor: kind::f16, A = B = bf16, D = f32, K-major A and B,
// M = 128, N = n (a multiple of 16: 128, or the real columns of the last site
// block rounded up)
__host__ __device__ constexpr uint32_t mma_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void arrive_local(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// bounded wait on an mbarrier phase that also gives up when another role of
// the CTA has aborted; returns false on abort or timeout (and then raises the
// CTA's abort flag and records the status)
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, unsigned long long limit,
                                           volatile int *abort_flag, int *status)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit) {
            *abort_flag = 1;
            atomicCAS(status, 0, FTWA_ERR_DEVICE_TIMEOUT);
            return false;
        }
    }
}

struct GemmArgs {
    const double *mu;      // [T][K]
    double *conn, *g2;     // [T][K][K]
    long long M;
    int K, n_kt, n_tiles, t0;
    int *status;
    unsigned long long timeout_ns;
};

struct GemmSmem {
    unsigned long long full[kStages], empty[kStages], accfull[2], accempty[2], drain;
    uint32_t tmem_base;
    int abort;
};

// one lane waits; the warp takes the decision together
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, unsigned long long limit,
                                          volatile int *abort_flag, int *status)
{
    bool got = false;
    if ((threadIdx.x & 31) == 0) got = wait_phase(bar, parity, limit, abort_flag, status);
    got = __shfl_sync(0xFFFFFFFFu, got ? 1 : 0, 0) != 0;
    return got;
}

// Epilogue warp (warp index w >= 2 of the CTA): adds columns 64 h .. 64 h + 63
// of tensor-memory lanes 32 (w % 4) .. +31 of accumulator `buf` (a finished
// 1024-sample segment) to its FP32 registers and releases the accumulator.
__device__ __forceinline__ bool drain_segment(float (&acc)[64], uint32_t d_tmem, int buf, long long seg, uint32_t accfull,
                                              uint32_t accempty, const GemmArgs &g, volatile int *abort_flag)
{
    const int warp = threadIdx.x >> 5, q = warp & 3, h = (warp - 2) >> 2;
    if (!warp_wait(accfull, (uint32_t)((seg / 2) & 1), g.timeout_ns, abort_flag, g.status)) return false;
    tmem_fence_after();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint32_t v[32];
        const uint32_t ta = d_tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * kTile + 64 * h + 32 * half);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
            "[%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(ta)
            : "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[32 * half + j] += __uint_as_float(v[j]);
    }
    tmem_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) arrive_local(accempty);
    return true;
}

// Epilogue output: conn (both triangles) and g2 of tile (kt, lt) at time t
__device__ __forceinline__ void write_tile(const float (&acc)[64], int t, int kt, int lt, const GemmArgs &g)
{
    const int warp = threadIdx.x >> 5, q = warp & 3, h = (warp - 2) >> 2;
    const int row = 32 * q + (threadIdx.x & 31);
    const bool same = kt == lt;
    const int k = kt * kTile + row;
    if (k >= g.K) return;
    const long long base = (long long)t * g.K * g.K;
    const double inv_m = 1.0 / (double)g.M;
    const double ok = g.mu[(long long)t * g.K + k] + 0.5;
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        const int l = lt * kTile + 64 * h + j;
        if (l >= g.K || (same && l < k)) continue;
        const double c = (double)acc[j] * inv_m;
        g.conn[base + (long long)k * g.K + l] = c;
        g.conn[base + (long long)l * g.K + k] = c;
        if (g.g2) {
            const double ol = g.mu[(long long)t * g.K + l] + 0.5;
            const double v = (c + ok * ol) / (ok * ol);
            g.g2[base + (long long)k * g.K + l] = v;
            g.g2[base + (long long)l * g.K + k] = v;
        }
    }
}

// MMA issue of one 64-sample chunk: 4 K-steps x {hi hi, hi lo, lo hi}
__device__ __forceinline__ void mma_chunk(uint32_t acc, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi, uint32_t b_lo,
                                          uint32_t idesc, bool first)
{
#pragma unroll
    for (int ks = 0; ks < kChunk / 16; ++ks) {
        const uint32_t ko = ks * 32;   // 16 bf16 = 32 bytes along K inside the swizzle atom
        const uint32_t acc0 = (!first || ks > 0) ? 1u : 0u;
        mma_bf16(acc, make_desc(a_hi + ko), make_desc(b_hi + ko), idesc, acc0);
        mma_bf16(acc, make_desc(a_hi + ko), make_desc(b_lo + ko), idesc, 1u);
        mma_bf16(acc, make_desc(a_lo + ko), make_desc(b_hi + ko), idesc, 1u);
    }
}

__global__ void __launch_bounds__(kThreadsG, 1) gram_tc_kernel(const __grid_constant__ CUtensorMap map_hi,
                                                               const __grid_constant__ CUtensorMap map_lo,
                                                               const GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand area: kStages x {A_hi, A_lo, B_hi, B_lo}
    unsigned char *img = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    GemmSmem *sh = reinterpret_cast<GemmSmem *>(img + kStages * 4 * kImage);
    volatile int *abort_flag = &sh->abort;

    const int tl = blockIdx.x / g.n_tiles, tile = blockIdx.x % g.n_tiles;
    int kt = 0, rem = tile;
    while (rem >= g.n_kt - kt) {
        rem -= g.n_kt - kt;
        ++kt;
    }
    const int lt = kt + rem;
    const bool same = kt == lt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n_chunks = (g.M + kChunk - 1) / kChunk;
    const long long n_seg = (n_chunks + kSegChunks - 1) / kSegChunks;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(smem_addr(&sh->full[i]), 1u);
            mbar_init(smem_addr(&sh->empty[i]), 1u);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_addr(&sh->accfull[i]), 1u);
            mbar_init(smem_addr(&sh->accempty[i]), (uint32_t)kEpiWarps);
        }
        mbar_init(smem_addr(&sh->drain), 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh->abort = 0;
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(&sh->tmem_base), 2 * kTile);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t d_tmem = sh->tmem_base;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            const uint32_t bytes = (same ? 2u : 4u) * (uint32_t)kImage;
            long long c = 0;
            for (; c < n_chunks; ++c) {
                const int st = (int)(c % kStages);
                if (c >= kStages &&
                    !wait_phase(smem_addr(&sh->empty[st]), (uint32_t)((c / kStages - 1) & 1), g.timeout_ns,
                                abort_flag, g.status))
                    break;
                const uint32_t fb = smem_addr(&sh->full[st]);
                const uint32_t base = smem_addr(img + st * 4 * kImage);
                const int x = (int)(c * kChunk);
                arrive_expect_tx(fb, bytes);
                tma_load_3d(base, &map_hi, x, kt * kTile, tl, fb);
                tma_load_3d(base + kImage, &map_lo, x, kt * kTile, tl, fb);
                if (!same) {
                    tma_load_3d(base + 2 * kImage, &map_hi, x, lt * kTile, tl, fb);
                    tma_load_3d(base + 3 * kImage, &map_lo, x, lt * kTile, tl, fb);
                }
            }
            if (*abort_flag) {
                // let the copies in flight land before the CTA exits
                for (long long d = (c > kStages ? c - kStages : 0); d < c; ++d) {
                    const uint64_t t0 = global_ns();
                    while (!mbar_try_wait_cluster(smem_addr(&sh->full[d % kStages]), (uint32_t)((d / kStages) & 1)) &&
                           global_ns() - t0 < g.timeout_ns) {
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            // columns of this tile: the real sites of the column block, rounded
            // up to 16 (the last block at K = 396 has 12)
            const int ncol = min(kTile, g.K - lt * kTile);
            const uint32_t idesc = mma_idesc((ncol + 15) / 16 * 16);
            bool ok = true;
            long long c = 0;
            for (long long seg = 0; seg < n_seg && ok; ++seg) {
                const int buf = (int)(seg & 1);
                if (seg >= 2 && !wait_phase(smem_addr(&sh->accempty[buf]), (uint32_t)((seg / 2 - 1) & 1),
                                            g.timeout_ns, abort_flag, g.status)) {
                    ok = false;
                    break;
                }
                tmem_fence_after();
                const uint32_t acc = d_tmem + (uint32_t)(buf * kTile);
                const long long c_end = (seg + 1) * kSegChunks < n_chunks ? (seg + 1) * kSegChunks : n_chunks;
                for (long long first = c; c < c_end; ++c) {
                    const int st = (int)(c % kStages);
                    if (!wait_phase(smem_addr(&sh->full[st]), (uint32_t)((c / kStages) & 1), g.timeout_ns,
                                    abort_flag, g.status)) {
                        ok = false;
                        break;
                    }
                    tmem_fence_after();
                    const uint32_t base = smem_addr(img + st * 4 * kImage);
                    const uint32_t a_hi = base, a_lo = base + kImage;
                    const uint32_t b_hi = same ? a_hi : base + 2 * kImage, b_lo = same ? a_lo : base + 3 * kImage;
                    mma_chunk(acc, a_hi, a_lo, b_hi, b_lo, idesc, c == first);
                    mma_commit(smem_addr(&sh->empty[st]));
                }
                if (ok) mma_commit(smem_addr(&sh->accfull[buf]));
            }
            // every issued MMA has completed before the accumulators are freed
            mma_commit(smem_addr(&sh->drain));
            const uint64_t t0 = global_ns();
            while (!mbar_try_wait_cluster(smem_addr(&sh->drain), 0u) && global_ns() - t0 < g.timeout_ns) {
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: segment sums and output ----------------
        // FP32 sum over segments: at most n_seg roundings of 2^-24, far below
        // the rounding of the 1024-sample tensor-core sums themselves
        float acc[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) acc[j] = 0.0f;
        bool ok = true;
        for (long long seg = 0; seg < n_seg && ok; ++seg) {
            const int buf = (int)(seg & 1);
            ok = drain_segment(acc, d_tmem, buf, seg, smem_addr(&sh->accfull[buf]), smem_addr(&sh->accempty[buf]), g,
                               abort_flag);
        }
        if (ok && *abort_flag == 0) write_tile(acc, g.t0 + tl, kt, lt, g);
    }

    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(d_tmem, 2 * kTile);
}

}  // namespace gram

// ---- host side -----------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

struct GramGeom {
    int K, Kd, n_kt, n_tiles, TB;   // Kd = max(K, 128) stored site rows
    long long Mp;
    size_t mu_bytes, ops_bytes;
};

// Times per batch: three waves of (time, tile) CTAs over the SMs (the tiles
// of the last, partly filled site block are cheaper; the hardware fills the
// SMs they free with the next CTAs), and at most about 6 GB of split operands.
GramGeom gram_geom(Plan *p, int64_t M, int32_t T)
{
    using namespace gram;
    GramGeom gg;
    gg.K = 2 * p->N;
    gg.n_kt = (gg.K + kTile - 1) / kTile;
    gg.Kd = std::max(gg.K, kTile);
    gg.n_tiles = gg.n_kt * (gg.n_kt + 1) / 2;
    gg.Mp = (M + kChunk - 1) / kChunk * kChunk;
    const size_t per_t = 2 * (size_t)gg.Kd * (size_t)gg.Mp * sizeof(__nv_bfloat16);
    const int sm = std::max(1, p->sm_count);
    int tb = std::max(1, 3 * sm / gg.n_tiles);
    tb = (int)std::min<size_t>((size_t)tb, std::max<size_t>(1, (size_t)(6ull << 30) / per_t));
    gg.TB = std::max(1, std::min(tb, (int)T));
    gg.mu_bytes = ((sizeof(double) * (size_t)T * gg.K + 255) / 256) * 256;
    gg.ops_bytes = per_t * gg.TB;
    return gg;
}

}  // namespace

int launch_gram_bf16x3(Plan *p, const void *snap, int64_t M, int32_t T, const double *mu, double *conn, double *g2,
                       cudaStream_t s)
{
    using namespace gram;
    if (p->precision != FTWA_FP32) return FTWA_ERR_UNSUPPORTED;   // the split is defined for FP32 snapshots
    if (M < 1 || T < 1) return FTWA_ERR_INVALID_ARGUMENT;
    if (M > (int64_t)0x7FFFFFFF - kChunk) return FTWA_ERR_UNSUPPORTED;   // TMA coordinates are 32-bit
    PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn();
    if (!encode) return FTWA_ERR_UNSUPPORTED;
    const GramGeom gg = gram_geom(p, M, T);
    GemmArgs a;
    a.mu = mu;
    a.conn = conn;
    a.g2 = g2;
    a.M = M;
    a.K = gg.K;
    a.n_kt = gg.n_kt;
    a.n_tiles = gg.n_tiles;
    a.status = p->d_status;
    a.timeout_ns = p->timeout_ns;
    const cuuint32_t estr[3] = {1, 1, 1};
    cudaError_t e;

    if (p->ws_bytes < gg.mu_bytes + gg.ops_bytes) return FTWA_ERR_OUT_OF_MEMORY;   // sized by the caller
    unsigned char *ws = reinterpret_cast<unsigned char *>(p->d_ws);
    __nv_bfloat16 *hi = reinterpret_cast<__nv_bfloat16 *>(ws + gg.mu_bytes);
    __nv_bfloat16 *lo = hi + gg.ops_bytes / (2 * sizeof(__nv_bfloat16));
    CUtensorMap map_hi, map_lo;
    // rows k >= Kd of the last tile's boxes read as zeros (TMA out-of-bounds fill)
    const cuuint64_t dims[3] = {(cuuint64_t)gg.Mp, (cuuint64_t)gg.Kd, (cuuint64_t)gg.TB};
    const cuuint64_t strides[2] = {(cuuint64_t)gg.Mp * 2, (cuuint64_t)gg.Kd * (cuuint64_t)gg.Mp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kChunk, (cuuint32_t)kTile, 1};
    for (int i = 0; i < 2; ++i) {
        CUresult r = encode(i == 0 ? &map_hi : &map_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, i == 0 ? (void *)hi : (void *)lo,
                            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return FTWA_ERR_CUDA;
    }
    const int smem = kStages * 4 * kImage + 1024 + (int)sizeof(GemmSmem);
    e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    for (int t0 = 0; t0 < T; t0 += gg.TB) {
        const int tb = std::min(gg.TB, T - t0);
        dim3 gs((unsigned)(gg.Mp / kChunk), (unsigned)((gg.Kd + kSplitSites - 1) / kSplitSites), (unsigned)tb);
        split_kernel<<<gs, 256, 0, s>>>(reinterpret_cast<const float *>(snap), mu, hi, lo, M, gg.K, gg.Kd, gg.Mp, t0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(e);
        a.t0 = t0;
        gram_tc_kernel<<<(unsigned)(tb * gg.n_tiles), kThreadsG, smem, s>>>(map_hi, map_lo, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return FTWA_OK;
}

size_t gram_bf16x3_workspace(Plan *p, const void *snap, int64_t M, int32_t T)
{
    const GramGeom gg = gram_geom(p, M, T);
    (void)snap;
    return gg.mu_bytes + gg.ops_bytes;
}

}  // namespace ftwa
