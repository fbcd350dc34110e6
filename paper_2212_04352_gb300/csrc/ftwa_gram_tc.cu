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
// One CTA per (time, 128x128 output tile of the upper triangle, sample
// split).  The CTA streams 64-sample chunks: all threads centre, split and
// write the operands as 128-byte-swizzled K-major images in shared memory
// (two stages), one thread issues the MMAs (M = N = 128, K = 16 per
// instruction) and commits them to an mbarrier.  The FP32 tile is written to
// a partial buffer; a second kernel sums the sample splits in FP64 and
// writes conn and g2.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "ftwa_internal.h"
#include "ptx.cuh"

namespace ftwa {

namespace gram {

constexpr int kTile = 128;          // output tile edge (features)
constexpr int kChunk = 64;          // samples per operand image (128 bytes of bf16)
constexpr int kImage = kTile * kChunk * 2;   // 16 KB per operand image
constexpr int kThreadsG = 256;

// byte offset of (row r, sample j) in a 128 x 64 bf16 K-major image with the
// 128-byte swizzle: 8-row atoms of 1024 bytes; 16-byte chunk c of row r sits
// at chunk position c ^ (r % 8)
__device__ __forceinline__ uint32_t swz(int r, int c16)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c16 ^ (r & 7)) << 4));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart
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
// M = 128, N = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTile >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct GramArgs {
    const float *X;        // [T][M][K]
    const double *mu;      // [T][K]
    float *partial;        // [splits][T][n_tiles][128][128]
    long long M;
    int K, T, n_kt, n_tiles, splits;
    long long chunks_per_split;
    int *status;
    unsigned long long timeout_ns;
};

// operand image of features [ft*128, ft*128+128) x samples [m0, m0+64)
__device__ __forceinline__ void build_image(const GramArgs &g, const float *Xt, const float *mu_f, int ft,
                                            long long m0, unsigned char *hi_img, unsigned char *lo_img)
{
    // item = (feature row r, 8-sample chunk c): lanes run over features so
    // every global load is coalesced across the warp
    for (int it = threadIdx.x; it < kTile * 8; it += kThreadsG) {
        const int r = it % kTile, c = it / kTile;
        const int k = ft * kTile + r;
        float y[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long long m = m0 + 8 * c + j;
            y[j] = (k < g.K && m < g.M) ? Xt[m * g.K + k] - mu_f[r] : 0.0f;
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 hb = __floats2bfloat162_rn(y[2 * j], y[2 * j + 1]);
            const float2 hf = __bfloat1622float2(hb);
            const __nv_bfloat162 lb = __floats2bfloat162_rn(y[2 * j] - hf.x, y[2 * j + 1] - hf.y);
            h[j] = *reinterpret_cast<const uint32_t *>(&hb);
            l[j] = *reinterpret_cast<const uint32_t *>(&lb);
        }
        const uint32_t off = swz(r, c);
        *reinterpret_cast<uint4 *>(hi_img + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(lo_img + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

__global__ void __launch_bounds__(kThreadsG, 1) gram_bf16x3_kernel(const GramArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned operand area: 2 stages x {A_hi, A_lo, B_hi, B_lo}
    unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *img = smem;                                        // 8 x 16 KB
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + 8 * kImage);   // 2 stage barriers
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);
    float *mu_a = reinterpret_cast<float *>(tmem_slot + 4);          // [128]
    float *mu_b = mu_a + kTile;                                       // [128]

    // tile index -> (t, kt <= lt, split)
    int idx = blockIdx.x;
    const int split = idx % g.splits;
    idx /= g.splits;
    const int tile = idx % g.n_tiles;
    const int t = idx / g.n_tiles;
    int kt = 0, rem = tile;
    while (rem >= g.n_kt - kt) {
        rem -= g.n_kt - kt;
        ++kt;
    }
    const int lt = kt + rem;
    const bool same = kt == lt;
    const float *Xt = g.X + (long long)t * g.M * g.K;
    const int warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bars[0]), 1u);
        mbar_init(smem_addr(&bars[1]), 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    for (int r = threadIdx.x; r < kTile; r += kThreadsG) {
        const int ka = kt * kTile + r, kb = lt * kTile + r;
        mu_a[r] = ka < g.K ? (float)g.mu[(long long)t * g.K + ka] : 0.0f;
        mu_b[r] = kb < g.K ? (float)g.mu[(long long)t * g.K + kb] : 0.0f;
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(tmem_slot), kTile);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t d_tmem = *tmem_slot;

    const long long c0 = (long long)split * g.chunks_per_split;
    const long long n_chunks_total = (g.M + kChunk - 1) / kChunk;
    const long long c1 = std::min<long long>(c0 + g.chunks_per_split, n_chunks_total);
    uint32_t phase[2] = {0u, 0u};
    bool issued[2] = {false, false};
    long long n_done = 0;
    for (long long c = c0; c < c1; ++c, ++n_done) {
        const int st = (int)(n_done & 1);
        unsigned char *a_hi = img + (st * 4 + 0) * kImage, *a_lo = img + (st * 4 + 1) * kImage;
        unsigned char *b_hi = same ? a_hi : img + (st * 4 + 2) * kImage;
        unsigned char *b_lo = same ? a_lo : img + (st * 4 + 3) * kImage;
        // the stage is free once the MMAs issued on it two chunks ago are done
        if (issued[st]) {
            if (threadIdx.x == 0 && !mbar_wait_bounded(smem_addr(&bars[st]), phase[st], g.timeout_ns)) {
                *abort_flag = 1;
                atomicCAS(g.status, 0, FTWA_ERR_DEVICE_TIMEOUT);
            }
            phase[st] ^= 1u;
            issued[st] = false;
            __syncthreads();
            if (*abort_flag) break;
            tmem_fence_after();
        }
        build_image(g, Xt, mu_a, kt, c * kChunk, a_hi, a_lo);
        if (!same) build_image(g, Xt, mu_b, lt, c * kChunk, b_hi, b_lo);
        fence_async_smem();
        tmem_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tmem_fence_after();
            const uint32_t sa_hi = smem_addr(a_hi), sa_lo = smem_addr(a_lo);
            const uint32_t sb_hi = smem_addr(b_hi), sb_lo = smem_addr(b_lo);
#pragma unroll
            for (int ks = 0; ks < kChunk / 16; ++ks) {
                const uint32_t ko = ks * 32;      // 16 bf16 = 32 bytes along K inside the swizzle atom
                const uint32_t acc0 = (n_done > 0 || ks > 0) ? 1u : 0u;
                mma_bf16(d_tmem, make_desc(sa_hi + ko), make_desc(sb_hi + ko), acc0);
                mma_bf16(d_tmem, make_desc(sa_hi + ko), make_desc(sb_lo + ko), 1u);
                mma_bf16(d_tmem, make_desc(sa_lo + ko), make_desc(sb_hi + ko), 1u);
            }
            mma_commit(smem_addr(&bars[st]));
        }
        issued[st] = true;
        __syncwarp();
    }
    // drain
    for (int st = 0; st < 2; ++st) {
        if (issued[st]) {
            if (threadIdx.x == 0 && !mbar_wait_bounded(smem_addr(&bars[st]), phase[st], g.timeout_ns)) {
                *abort_flag = 1;
                atomicCAS(g.status, 0, FTWA_ERR_DEVICE_TIMEOUT);
            }
        }
    }
    __syncthreads();
    tmem_fence_after();

    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows) and
    // columns 64 (w / 4) .. +63; an empty split writes zeros
    const int row = 32 * (warp & 3) + (threadIdx.x & 31);
    const int col0 = 64 * (warp >> 2);
    float *out = g.partial + ((((long long)split * g.T + t) * g.n_tiles + tile) * kTile + row) * kTile + col0;
    const bool have = n_done > 0 && *abort_flag == 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t v[32];
        const uint32_t ta = d_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(col0 + 32 * h);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(ta)
            : "memory");
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
            float4 f;
            f.x = have ? __uint_as_float(v[j]) : 0.0f;
            f.y = have ? __uint_as_float(v[j + 1]) : 0.0f;
            f.z = have ? __uint_as_float(v[j + 2]) : 0.0f;
            f.w = have ? __uint_as_float(v[j + 3]) : 0.0f;
            *reinterpret_cast<float4 *>(out + 32 * h + j) = f;
        }
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(d_tmem, kTile);
}

// Sum the sample splits in FP64 and write conn (both triangles) and g2.
__global__ void gram_reduce_kernel(const float *partial, int splits, int T, int n_kt, int n_tiles, int K, long long M,
                                   const double *mu, double *conn, double *g2)
{
    const long long total = (long long)T * n_tiles * kTile * kTile;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(i % kTile), row = (int)((i / kTile) % kTile);
        const int tile = (int)((i / ((long long)kTile * kTile)) % n_tiles);
        const int t = (int)(i / ((long long)kTile * kTile * n_tiles));
        int kt = 0, rem = tile;
        while (rem >= n_kt - kt) {
            rem -= n_kt - kt;
            ++kt;
        }
        const int lt = kt + rem;
        const int k = kt * kTile + row, l = lt * kTile + col;
        if (k >= K || l >= K) continue;
        if (kt == lt && l < k) continue;          // diagonal tile: each pair once
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += (double)partial[(((long long)sp * T + t) * n_tiles + tile) * kTile * kTile +
                                                               (long long)row * kTile + col];
        const double c = s / (double)M;
        const long long base = (long long)t * K * K;
        conn[base + (long long)k * K + l] = c;
        conn[base + (long long)l * K + k] = c;
        if (g2) {
            const double ok = mu[(long long)t * K + k] + 0.5, ol = mu[(long long)t * K + l] + 0.5;
            const double v = (c + ok * ol) / (ok * ol);
            g2[base + (long long)k * K + l] = v;
            g2[base + (long long)l * K + k] = v;
        }
    }
}

}  // namespace gram

// Sample splits: enough CTAs to fill the machine twice, and every split's
// FP32 tensor-memory accumulation limited to kMaxChunksPerSplit chunks (1024
// samples), so that the FP32 rounding of a long same-sign sum (the
// variances) stays far below the sampling error; splits are summed in FP64.
static void gram_splits(Plan *p, long long n_chunks, long long base_ctas, long long &splits, long long &cps)
{
    constexpr long long kMaxChunksPerSplit = 16;
    splits = std::max<long long>(1, (2LL * std::max(1, p->sm_count) + base_ctas - 1) / base_ctas);
    splits = std::min<long long>(splits, std::max<long long>(1, n_chunks / 4));
    splits = std::max<long long>(splits, (n_chunks + kMaxChunksPerSplit - 1) / kMaxChunksPerSplit);
    cps = (n_chunks + splits - 1) / splits;
    splits = (n_chunks + cps - 1) / cps;
}

int launch_gram_bf16x3(Plan *p, const void *snap, int64_t M, int32_t T, const double *mu, double *conn, double *g2,
                       cudaStream_t s)
{
    using namespace gram;
    if (p->precision != FTWA_FP32) return FTWA_ERR_UNSUPPORTED;   // the split is defined for FP32 snapshots
    const int K = 2 * p->N;
    const int n_kt = (K + kTile - 1) / kTile;
    const int n_tiles = n_kt * (n_kt + 1) / 2;
    const long long n_chunks = (M + kChunk - 1) / kChunk;
    const long long base_ctas = (long long)T * n_tiles;
    long long splits, cps;
    gram_splits(p, n_chunks, base_ctas, splits, cps);
    // workspace: mu already occupies the first T*K doubles
    const size_t mu_bytes = ((sizeof(double) * (size_t)T * K + 255) / 256) * 256;
    const size_t part_bytes = sizeof(float) * (size_t)splits * T * n_tiles * kTile * kTile;
    if (p->ws_bytes < mu_bytes + part_bytes) return FTWA_ERR_OUT_OF_MEMORY;   // sized by the caller below
    float *partial = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(p->d_ws) + mu_bytes);
    GramArgs g;
    g.X = reinterpret_cast<const float *>(snap);
    g.mu = mu;
    g.partial = partial;
    g.M = M;
    g.K = K;
    g.T = T;
    g.n_kt = n_kt;
    g.n_tiles = n_tiles;
    g.splits = (int)splits;
    g.chunks_per_split = cps;
    g.status = p->d_status;
    g.timeout_ns = p->timeout_ns;
    const int smem = 8 * kImage + 1024 + 64 + 2 * kTile * 4 + 64;
    cudaError_t e = cudaFuncSetAttribute(gram_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    gram_bf16x3_kernel<<<(unsigned)(base_ctas * splits), kThreadsG, smem, s>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e);
    const long long total = (long long)T * n_tiles * kTile * kTile;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 65535LL * 8);
    gram_reduce_kernel<<<blocks, 256, 0, s>>>(partial, (int)splits, T, n_kt, n_tiles, K, M, mu, conn, g2);
    return set_cuda_error(cudaGetLastError());
}

size_t gram_bf16x3_workspace(Plan *p, int64_t M, int32_t T)
{
    using namespace gram;
    const int K = 2 * p->N;
    const int n_kt = (K + kTile - 1) / kTile;
    const int n_tiles = n_kt * (n_kt + 1) / 2;
    const long long n_chunks = (M + kChunk - 1) / kChunk;
    const long long base_ctas = (long long)T * n_tiles;
    long long splits, cps;
    gram_splits(p, n_chunks, base_ctas, splits, cps);
    const size_t mu_bytes = ((sizeof(double) * (size_t)T * K + 255) / 256) * 256;
    return mu_bytes + sizeof(float) * (size_t)splits * T * n_tiles * kTile * kTile;
}

}  // namespace ftwa
