// Tiled persistent RK4 stepper for FP32 states (Eq. 6, on-site U).
//
// Same method and arithmetic as the banded stepper (Eq. 6 with classical
// RK4; the stage state in shared memory, double-buffered; y0 and the stage
// accumulator in tensor memory; a thread-block cluster per sample for large
// lattices), with a layout chosen so that the inner loop is almost free of
// integer work:
//  - Shared memory is block-major: for each 31-column block b and spin s, the
//    rows of this rank are stored at a fixed stride of 248 B (one complex
//    FP32 value per lane, lanes 0..30; lane 31 idles), element (s, p, q) at
//    Z(s, b) + 248 p + 8 lane(q).  Row offsets inside a tile are therefore
//    immediates of the load, and since 248 B is 31 bank pairs, the elements
//    of one column in 16 consecutive rows (the mirror-band stores of a row)
//    fall in 16 distinct bank pairs.  Regions, slots and stage buffers start
//    on 128-byte boundaries, so a row's bank pattern is the lane's.
//  - Each row stores the upper triangle plus a mirror band of bw entries
//    below the diagonal (bw = lattice bandwidth), as in the banded stepper,
//    so every read of Eq. 6 is a direct load.  Empty neighbour slots read
//    the lane's own element with a zero hopping.
//  - A tile is up to kR consecutive rows of one spin and one column block.
//    A lane owns column q of the tile; the row-part gathers rho_pk,
//    k in nb(q), are at fixed byte offsets from the lane's own element for
//    every row of the rank (one table entry per block and lane), and the
//    column-part reads rho_kq, k in nb(p), at per-row offsets (k - p) 248
//    held with the row's hoppings in a per-rank table in shared memory.
//  - On lattices whose site order has every site's neighbours among p - 1,
//    p + 1 and at most one other site (honeycomb flakes numbered along
//    rows), the column-part values of rows p -+ 1 are the lane's own values
//    of the neighbouring rows of the tile, carried in registers.
// Per element (p, q), p <= q, spin s (Eq. 6):
//   k_pq = i [ sum_{k in nb(q)} t_qk rho_pk - sum_{k in nb(p)} t_pk rho_kq
//              + U (Re rho_pp,sbar - Re rho_qq,sbar) rho_pq ].
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <vector>

#include <new>

#include "ftwa_internal.h"
#include "ptx.cuh"

namespace ftwa {
namespace tile {

constexpr int kR = 8;                     // rows per tile
// tensor-memory columns per warp: warps w, w + 4, ... share lane quadrant w % 4
// and split the 512 columns (multiples of 8 for the 8-column row-pair blocks)
__host__ __device__ constexpr int cols_per_warp(int warps) { return (512 / (warps / 4)) / 8 * 8; }
constexpr int kW = 31;                    // columns per block (lanes 0..30; lane 31 idle)
constexpr int kMaxBlk = (FTWA_MAX_SITES + kW - 1) / kW;
constexpr int kRowBytes = 8 * kW;         // one row of a block: 248 B, so consecutive rows of a
                                          // column fall in distinct bank pairs
constexpr int kIdleQ = -(1 << 20);        // column of the idle lane: fails every element predicate

struct TileHeader {
    unsigned long long dead_bar;  // never completes (timeout test hook)
    uint32_t tmem_base;
    int abort;
    int item;                     // batched launch: the cluster's current work item
};

extern __shared__ __align__(16) unsigned char tile_smem[];

// Column-part data of one spin-row (one entry per spin-row, written from the
// owning rank's point of view; each rank copies its rows into shared memory).
struct __align__(16) RowEntry {
    float mt[3];      // -t_pk of the three column-part slots (0: empty slot)
    uint32_t flags;   // bit n: slot n is in another rank; bit 3 + n: that rank is the next one
    int32_t dcol[3];  // local slot: (k - p) * 248 (0 for an empty slot); remote slot: k * 248
    int32_t mir;      // Z(s, blk(p)) + 8 lane(p): element (q, p) is at mir + 248 q
};

// Lattices with carried rows p -+ 1: the same 32 bytes per spin-row, with the
// hoppings as (h, h) pairs for packed FMAs.
struct __align__(16) RowPm1 {
    float m0[2];      // -t of row p - 1 (0: absent)
    float m1[2];      // -t of row p + 1
    float m2[2];      // -t of the far neighbour k (0: none)
    int32_t far;      // local: (k - p) * 248; another rank: k * 248 | 1, | 2 when it is the next rank
    int32_t mir;      // as RowEntry::mir
};
static_assert(sizeof(RowPm1) == sizeof(RowEntry), "row tables share one slot size");

// Tile descriptor: x = p0 | cnt << 9 | b << 13 | slot << 17 (p0 a spin-row);
// y = flags below.
enum : uint32_t {
    kDiag = 1u,        // a row's diagonal element lies in the tile
    kBand = 2u,        // some lane holds a mirror-band element (0 < q - p <= bw)
    kPrevShift = 3,    // 2 bits: row p0 - 1 is 0 local, 1 absent (zero hopping), 2 in the previous rank
    kNextShift = 5,    // 2 bits: row p0 + cnt is 0 local, 1 absent (zero hopping), 2 in the next rank
    kRemote = 128u,    // some row of the tile reads a column-part slot of another rank
    kRemoteMir = 256u, // some mirror-band row of the tile may belong to the next rank
    kFull = 512u,      // carried-row lattice, kR rows, no kRemoteMir, far slots of at most one
                       // other rank: the unrolled path
    kFarNext = 1024u,  // kFull tile whose remote far slots are in the next rank
};

struct TileArgs {
    int N, C, S, nblk, qoff, bw, warps, pm1;
    int slot_bytes, buf_bytes;       // one slot of one stage buffer; one stage buffer
    int k_tiles;                     // tile entries per warp
    float U, dt;
    long long M, n_steps;
    int out_every;
    float2 *rho;                     // [M][2][N][N]
    float *snap;                     // [n_out][M][2N] or null
    int *status;
    unsigned long long timeout_ns;
    int force_timeout;
    int row_begin[kMaxCluster + 1];  // spin-rows of each rank
    int zoff[kMaxCluster][2][kMaxBlk];   // Z(s, b) of each rank (byte offset inside a slot)
    const uint2 *tiles;              // [C][warps][k_tiles]
    const int4 *koff;                // [C][nblk][32] row-part byte offsets of the three slots
    const float2 *tq;                // [nblk][32][3] (t, t) of the row-part slots
    const RowEntry *rows;            // [2N]
    int rows_bytes;                  // shared-memory bytes of the largest rank's row table
};

// ---- address arithmetic shared by the kernel and the host layout check --------
__host__ __device__ __forceinline__ int blk_of(int q, int qoff) { return (q - qoff) / kW; }
__host__ __device__ __forceinline__ int lane_of(int q, int qoff) { return (q - qoff) % kW; }
__host__ __device__ __forceinline__ int td_p0(uint32_t x) { return x & 511; }
__host__ __device__ __forceinline__ int td_cnt(uint32_t x) { return (x >> 9) & 15; }
__host__ __device__ __forceinline__ int td_blk(uint32_t x) { return (x >> 13) & 15; }
__host__ __device__ __forceinline__ int td_slot(uint32_t x) { return (x >> 17) & 255; }
__host__ __device__ __forceinline__ uint32_t td_make(int p0, int cnt, int b, int slot)
{
    return (uint32_t)p0 | ((uint32_t)cnt << 9) | ((uint32_t)b << 13) | ((uint32_t)slot << 17);
}
// byte offset (inside a slot) of element (s, p, q) in a rank whose origins are z
__host__ __device__ __forceinline__ int elem_off(const int (*z)[kMaxBlk], int s, int p, int q, int qoff)
{
    return z[s][blk_of(q, qoff)] + kRowBytes * p + 8 * lane_of(q, qoff);
}

// ---- device helpers ------------------------------------------------------------
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float2 ld_cluster(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster(uint32_t a, float2 v)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
// tensor memory: a row pair's y0 and acc (8 words: y0 a, y0 b, acc a, acc b)
__device__ __forceinline__ void tm_ld8(uint32_t ta, uint32_t (&w)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "r"(ta));
}
__device__ __forceinline__ void tm_wait8(uint32_t (&w)[8])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]), "+r"(w[6]), "+r"(w[7]));
}
__device__ __forceinline__ void tm_st4(uint32_t ta, float2 a, float2 b)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ta),
                 "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(b.x)),
                 "r"(__float_as_uint(b.y)));
}
// y0 of a row pair and a zeroed accumulator (all 8 words)
__device__ __forceinline__ void tm_st8z(uint32_t ta, float2 a, float2 b)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta),
                 "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(b.x)),
                 "r"(__float_as_uint(b.y)), "r"(0u), "r"(0u), "r"(0u), "r"(0u));
}

template <bool CLUSTER>
__device__ __forceinline__ void stage_sync()
{
    if constexpr (CLUSTER) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        __syncthreads();
    }
}

struct TileCtx {
    uint32_t smem_s;          // shared::cta address of the dynamic shared memory
    int buf0;                 // byte offset of stage buffer 0
    int diag_off;             // byte offset of the diagonals [2 buffers][S][2N] (float)
    int rows_off;             // byte offset of this rank's row table
    int rb0, rb1;             // this rank's spin-rows
    uint32_t diag_s;
    uint32_t prev_c, next_c;  // shared::cluster address of smem in the previous / next rank
    int rank;                 // rank inside the problem's group of a.C CTAs
    uint32_t rank_base;       // cluster rank of that group's first CTA
    const uint2 *tiles;
    uint32_t t_state;
    int lane;
};

// The lanes holding a row's diagonal publish its new value to every rank's
// diagonal table (and, after the final stage, to the snapshot).
template <bool FINAL, bool CLUSTER>
__device__ __forceinline__ void publish_diag(const TileArgs &a, const TileCtx &c, bool mine, int cur, int slot, int s,
                                             int q, float dnew, long long b_id, bool snap_now, long long snap_row)
{
    if (!mine) return;
    const int twoN = 2 * a.N;
    const int di = ((cur ^ 1) * a.S + slot) * twoN + s * a.N + q;
    if constexpr (CLUSTER) {
        const uint32_t da = c.diag_s + (uint32_t)(4 * di);
        for (int r = 0; r < a.C; ++r) {
            const uint32_t ra = map_rank(da, c.rank_base + (uint32_t)r);
            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(dnew) : "memory");
        }
    } else {
        *reinterpret_cast<float *>(tile_smem + c.diag_off + 4 * di) = dnew;
    }
    if (FINAL && snap_now) {
        const long long m = b_id * a.S + slot;
        if (m < a.M) a.snap[(snap_row * a.M + m) * twoN + s * a.N + q] = dnew;
    }
}

// One RK4 stage over the rows of one tile.  Stage buffer sc.cur holds the
// stage state; the next stage state goes to the other buffer.  Stages 0-2
// share one code path: the stage accumulator starts each step at zero (the
// final stage stores zeros), acc += b k and the next stage state is
// y0 + cc k, with (b, cc) = (1, dt/2), (2, dt/2), (2, dt); the final stage
// forms y0 + dt/6 (acc + k).  Everything that depends only on the lane
// (column) or only on the tile is formed once per tile; the rare cases (the
// diagonal, the mirror band, rows of another rank) are warp-uniform branches
// or per-lane predicates on values formed per tile.
struct StageC {
    int cur;     // stage buffer holding the stage state
    float b;     // weight of k in the accumulator
    float cc;    // next stage state: y0 + cc k
};

__device__ __forceinline__ float4 lds128(int off) { return *reinterpret_cast<const float4 *>(tile_smem + off); }

// far column-part value: a shared-memory load of this CTA or, where `rem` is
// set, a distributed shared-memory load of a peer (both predicated, no branch)
__device__ __forceinline__ float2 ld_far(uint32_t local_addr, uint32_t remote_addr, uint32_t rem)
{
    float2 v;
    asm volatile(
        "{\n\t.reg .pred pr;\n\tsetp.ne.u32 pr, %3, 0;\n\t"
        "@pr ld.shared::cluster.v2.f32 {%0, %1}, [%4];\n\t"
        "@!pr ld.shared.v2.f32 {%0, %1}, [%2];\n\t}"
        : "=f"(v.x), "=f"(v.y)
        : "r"(local_addr), "r"(rem), "r"(remote_addr));
    return v;
}

template <bool FINAL, bool PM1, bool CLUSTER>
__device__ __forceinline__ void tile_rows(const TileArgs &a, const TileCtx &c, const StageC &sc, uint2 td, int e_base,
                                          long long b_id, bool snap_now, long long snap_row)
{
    const int cur = FINAL ? 1 : sc.cur;
    const int N = a.N, twoN = 2 * N, lane = c.lane;
    const int p0 = td_p0(td.x), cnt = td_cnt(td.x), blk = td_blk(td.x), slot = td_slot(td.x);
    const bool diag_t = (td.y & kDiag) != 0, band_t = (td.y & kBand) != 0, rmir_t = (td.y & kRemoteMir) != 0;
    const int s = p0 >= N ? 1 : 0;
    const int pp0 = p0 - s * N;                       // site index of row 0 of the tile
    const int la = lane < kW ? lane : kW - 1;           // the idle lane shadows lane 30's addresses
    const int c0 = a.qoff + kW * blk;
    const int q = lane < kW ? c0 + lane : kIdleQ;
    const int qc = q < 0 ? 0 : q;
    const int slot_off = slot * a.slot_bytes;
    const int cur_off = c.buf0 + cur * a.buf_bytes + slot_off;
    const int dnext = (cur ? -1 : 1) * a.buf_bytes;   // next stage buffer minus this one
    const int own0 = cur_off + a.zoff[c.rank][s][blk] + kRowBytes * pp0 + 8 * la;   // element (p0, q)
    const int4 ko = __ldg(&a.koff[(c.rank * a.nblk + blk) * 32 + lane]);
    const float2 *tqp = a.tq + (blk * 32 + lane) * 3;
    const float2 tq0 = __ldg(tqp), tq1 = __ldg(tqp + 1), tq2 = __ldg(tqp + 2);
    const int dg_off = c.diag_off + 4 * ((cur * a.S + slot) * twoN + (1 - s) * N);   // other spin's diagonal
    auto lds = [&](int off) -> float2 { return *reinterpret_cast<const float2 *>(tile_smem + off); };
    auto ldf = [&](int off) -> float { return *reinterpret_cast<const float *>(tile_smem + off); };
    auto sts = [&](int off, float2 v) { *reinterpret_cast<float2 *>(tile_smem + off) = v; };
    const float uq = a.U * ldf(dg_off + 4 * qc);
    const float sdt = a.dt * (1.0f / 6.0f);
    const int rt0 = c.rows_off + (int)sizeof(RowEntry) * (p0 - c.rb0);
    // cluster-space addresses of (row 0, column q) in the previous / next rank's current buffer
    uint32_t base_prev = 0, base_next = 0;
    if constexpr (CLUSTER) {
        if (c.rank > 0) base_prev = c.prev_c + (uint32_t)(cur_off + a.zoff[c.rank - 1][s][blk] + 8 * la);
        if (c.rank + 1 < a.C) base_next = c.next_c + (uint32_t)(cur_off + a.zoff[c.rank + 1][s][blk] + 8 * la);
    }
    // mirror band: row q of this rank, or of the next one
    const bool mir_local = s * N + q < c.rb1;
    const int mir_lane = kRowBytes * q + cur_off + dnext;
    float dnew = 0.f;                                 // this lane's new diagonal value (q == p)

    // carried column-part values (PM1): rows p0 - 1 and p0 + cnt of the tile
    float2 vprev = make_float2(0.f, 0.f), vcur = make_float2(0.f, 0.f), vlast = make_float2(0.f, 0.f);
    if constexpr (PM1) {
        const uint32_t pk = (td.y >> kPrevShift) & 3, nk = (td.y >> kNextShift) & 3;
        if (CLUSTER && pk == 2) vprev = ld_cluster(base_prev + (uint32_t)(kRowBytes * (pp0 - 1)));
        else vprev = lds(pk == 0 ? own0 - kRowBytes : own0);          // absent: a finite value, zero hopping
        if (CLUSTER && nk == 2) vlast = ld_cluster(base_next + (uint32_t)(kRowBytes * (pp0 + cnt)));
        else vlast = lds(nk == 0 ? own0 + kRowBytes * cnt : own0);
        vcur = lds(own0);
    }

    auto row = [&](int i, float2 &y0, float2 &acc) {
        const int p = pp0 + i;
        const int own = own0 + kRowBytes * i;
        float2 ov;
        float2 h = make_float2(0.f, 0.f);
        int mir;
        // + sum_{k in nb(q)} t_qk rho_pk (row p)
        h = ffma2(tq0, lds(own + ko.x), h);
        h = ffma2(tq1, lds(own + ko.y), h);
        h = ffma2(tq2, lds(own + ko.z), h);
        // - sum_{k in nb(p)} t_pk rho_kq (column q)
        if constexpr (PM1) {
            const float4 m01 = lds128(rt0 + (int)sizeof(RowPm1) * i);
            const float4 m2f = lds128(rt0 + (int)sizeof(RowPm1) * i + 16);
            const int far = __float_as_int(m2f.z);
            mir = __float_as_int(m2f.w);
            ov = vcur;
            const bool in_tile = i + 1 < cnt;
            const float2 vn = lds(in_tile ? own + kRowBytes : own);
            const float2 vnext = in_tile ? vn : vlast;
            float2 vf;
            if (CLUSTER && (far & 1)) vf = ld_cluster(((far & 2) ? base_next : base_prev) + (uint32_t)(far & ~3));
            else vf = lds(own + far);
            h = ffma2(make_float2(m01.x, m01.y), vprev, h);
            h = ffma2(make_float2(m01.z, m01.w), vnext, h);
            h = ffma2(make_float2(m2f.x, m2f.y), vf, h);
            vprev = vcur;
            vcur = vnext;
        } else {
            const RowEntry re = *reinterpret_cast<const RowEntry *>(tile_smem + rt0 + (int)sizeof(RowEntry) * i);
            mir = re.mir;
            ov = lds(own);
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                float2 v;
                if (CLUSTER && (re.flags & (1u << n)))
                    v = ld_cluster((((re.flags >> (3 + n)) & 1u) ? base_next : base_prev) + (uint32_t)re.dcol[n]);
                else
                    v = lds(own + re.dcol[n]);
                h.x = fmaf(re.mt[n], v.x, h.x);
                h.y = fmaf(re.mt[n], v.y, h.y);
            }
        }
        // + U (Re rho_pp,sbar - Re rho_qq,sbar) rho_pq
        const float coef = fmaf(a.U, ldf(dg_off + 4 * p), -uq);
        h.x = fmaf(coef, ov.x, h.x);
        h.y = fmaf(coef, ov.y, h.y);
        // k = i h; the diagonal of Eq. 6 is real (the imaginary part is rounding residue)
        const float kx = -h.y;
        const float ky = q == p ? 0.f : h.x;
        float2 nx;
        if constexpr (!FINAL) {
            acc.x = fmaf(sc.b, kx, acc.x);
            acc.y = fmaf(sc.b, ky, acc.y);
            nx.x = fmaf(sc.cc, kx, y0.x);
            nx.y = fmaf(sc.cc, ky, y0.y);
        } else {
            nx.x = fmaf(sdt, acc.x + kx, y0.x);
            nx.y = fmaf(sdt, acc.y + ky, y0.y);
            y0 = nx;
        }
        if (q >= p) sts(own + dnext, nx);
        if (q == p) dnew = nx.x;
        if (band_t) {
            // mirror entry (q, p) = conj(rho_pq) in row q, for 0 < q - p <= bw
            const bool mb = (unsigned)(q - p - 1) < (unsigned)a.bw;
            const float2 cj = make_float2(nx.x, -nx.y);
            if (!rmir_t) {
                if (mb) sts(mir + mir_lane, cj);
            } else if (mb) {
                if (mir_local) {
                    sts(mir + mir_lane, cj);
                } else {
                    const int bp = blk_of(p, a.qoff);
                    const int mn = mir - a.zoff[c.rank][s][bp] + a.zoff[c.rank + 1][s][bp];
                    st_cluster(c.next_c + (uint32_t)(mn + mir_lane), cj);
                }
            }
        }
    };

    uint32_t w[8];
    tm_ld8(c.t_state + (uint32_t)(8 * e_base), w);
    for (int i = 0; i < cnt; i += 2) {
        tm_wait8(w);
        float2 y0a = make_float2(__uint_as_float(w[0]), __uint_as_float(w[1]));
        float2 y0b = make_float2(__uint_as_float(w[2]), __uint_as_float(w[3]));
        float2 acca = make_float2(__uint_as_float(w[4]), __uint_as_float(w[5]));
        float2 accb = make_float2(__uint_as_float(w[6]), __uint_as_float(w[7]));
        row(i, y0a, acca);
        if (i + 1 < cnt) row(i + 1, y0b, accb);
        const uint32_t ta = c.t_state + (uint32_t)(8 * (e_base + (i >> 1)));
        if constexpr (!FINAL) tm_st4(ta + 4, acca, accb);
        else tm_st8z(ta, y0a, y0b);
        if (i + 2 < cnt) tm_ld8(ta + 8, w);
    }
    publish_diag<FINAL, CLUSTER>(a, c, diag_t && q >= pp0 && q < pp0 + cnt, cur, slot, s, q, dnew, b_id, snap_now,
                                 snap_row);
}

// Full tiles of lattices with carried rows p -+ 1 (kR = 8 rows, no mirror
// row in another rank): the row loop unrolled, every row offset an immediate
// of its load, no per-row branch.  REMOTE: the far column-part slot of some
// row is in another rank (a predicated pair of loads per row).
template <bool FINAL, bool CLUSTER, bool REMOTE>
__device__ __forceinline__ void tile_rows8(const TileArgs &a, const TileCtx &c, const StageC &sc, uint2 td, int e_base,
                                           long long b_id, bool snap_now, long long snap_row)
{
    const int cur = FINAL ? 1 : sc.cur;
    const int N = a.N, twoN = 2 * N, lane = c.lane;
    const int p0 = td_p0(td.x), blk = td_blk(td.x), slot = td_slot(td.x);
    const bool diag_t = (td.y & kDiag) != 0, band_t = (td.y & kBand) != 0;
    const int s = p0 >= N ? 1 : 0;
    const int pp0 = p0 - s * N;
    const int la = lane < kW ? lane : kW - 1;
    const int q = lane < kW ? a.qoff + kW * blk + lane : kIdleQ;
    const int qi = q - pp0;                           // tile row holding this lane's diagonal
    const int qc = q < 0 ? 0 : q;
    const int cur_off = c.buf0 + cur * a.buf_bytes + slot * a.slot_bytes;
    const int dnext = (cur ? -1 : 1) * a.buf_bytes;
    const int own0 = cur_off + a.zoff[c.rank][s][blk] + kRowBytes * pp0 + 8 * la;
    const int4 ko = __ldg(&a.koff[(c.rank * a.nblk + blk) * 32 + lane]);
    const float2 *tqp = a.tq + (blk * 32 + lane) * 3;
    const float2 tq0 = __ldg(tqp), tq1 = __ldg(tqp + 1), tq2 = __ldg(tqp + 2);
    const int dg = c.diag_off + 4 * ((cur * a.S + slot) * twoN + (1 - s) * N);
    auto lds = [&](int off) -> float2 { return *reinterpret_cast<const float2 *>(tile_smem + off); };
    auto ldf = [&](int off) -> float { return *reinterpret_cast<const float *>(tile_smem + off); };
    auto sts = [&](int off, float2 v) { *reinterpret_cast<float2 *>(tile_smem + off) = v; };
    const float uq = a.U * ldf(dg + 4 * qc);
    const int dg0 = dg + 4 * pp0;
    const float sdt = a.dt * (1.0f / 6.0f);
    const int rt0 = c.rows_off + (int)sizeof(RowPm1) * (p0 - c.rb0);
    const int mir_lane = kRowBytes * q + cur_off + dnext;
    const int r0 = own0 + ko.x, r1 = own0 + ko.y, r2 = own0 + ko.z;
    uint32_t base_far = 0;   // (row 0, column q) in the rank holding the tile's remote far slots
    float2 vprev, vlast;
    {
        uint32_t base_prev = 0, base_next = 0;
        if constexpr (CLUSTER) {
            if (c.rank > 0) base_prev = c.prev_c + (uint32_t)(cur_off + a.zoff[c.rank - 1][s][blk] + 8 * la);
            if (c.rank + 1 < a.C) base_next = c.next_c + (uint32_t)(cur_off + a.zoff[c.rank + 1][s][blk] + 8 * la);
        }
        base_far = (td.y & kFarNext) ? base_next : base_prev;
        const uint32_t pk = (td.y >> kPrevShift) & 3, nk = (td.y >> kNextShift) & 3;
        if (CLUSTER && pk == 2) vprev = ld_cluster(base_prev + (uint32_t)(kRowBytes * (pp0 - 1)));
        else vprev = lds(pk == 0 ? own0 - kRowBytes : own0);
        if (CLUSTER && nk == 2) vlast = ld_cluster(base_next + (uint32_t)(kRowBytes * (pp0 + kR)));
        else vlast = lds(nk == 0 ? own0 + kRowBytes * kR : own0);
    }
    float2 vcur = lds(own0);
    float dnew = 0.f;
    const uint32_t t0 = c.t_state + (uint32_t)(8 * e_base);
    const uint32_t own0_s = c.smem_s + (uint32_t)own0;

    // row pairs: unrolled, except in tiles with remote far slots (register
    // budget at 768 threads)
#pragma unroll(REMOTE ? 1 : kR / 2)
    for (int j = 0; j < kR / 2; ++j) {
        uint32_t w[8];
        tm_ld8(t0 + 8 * j, w);
        tm_wait8(w);
        float2 y0[2] = {make_float2(__uint_as_float(w[0]), __uint_as_float(w[1])),
                        make_float2(__uint_as_float(w[2]), __uint_as_float(w[3]))};
        float2 acc[2] = {make_float2(__uint_as_float(w[4]), __uint_as_float(w[5])),
                         make_float2(__uint_as_float(w[6]), __uint_as_float(w[7]))};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int i = 2 * j + u;
            const int own = own0 + kRowBytes * i;
            const float4 m01 = lds128(rt0 + (int)sizeof(RowPm1) * i);
            const float4 m2f = lds128(rt0 + (int)sizeof(RowPm1) * i + 16);
            const int far = __float_as_int(m2f.z);
            float2 h = make_float2(0.f, 0.f);
            h = ffma2(tq0, lds(r0 + kRowBytes * i), h);
            h = ffma2(tq1, lds(r1 + kRowBytes * i), h);
            h = ffma2(tq2, lds(r2 + kRowBytes * i), h);
            const float2 vnext = i + 1 < kR ? lds(own + kRowBytes) : vlast;
            float2 vf;
            if constexpr (REMOTE && CLUSTER) {
                const uint32_t ra = base_far + (uint32_t)(far & ~3);
                vf = ld_far(own0_s + (uint32_t)(kRowBytes * i + far), ra, (uint32_t)(far & 1));
            } else {
                vf = lds(own + far);
            }
            h = ffma2(make_float2(m01.x, m01.y), vprev, h);
            h = ffma2(make_float2(m01.z, m01.w), vnext, h);
            h = ffma2(make_float2(m2f.x, m2f.y), vf, h);
            const float coef = fmaf(a.U, ldf(dg0 + 4 * i), -uq);
            h.x = fmaf(coef, vcur.x, h.x);
            h.y = fmaf(coef, vcur.y, h.y);
            const float kx = -h.y;
            const float ky = qi == i ? 0.f : h.x;
            float2 nx;
            if constexpr (!FINAL) {
                acc[u].x = fmaf(sc.b, kx, acc[u].x);
                acc[u].y = fmaf(sc.b, ky, acc[u].y);
                nx.x = fmaf(sc.cc, kx, y0[u].x);
                nx.y = fmaf(sc.cc, ky, y0[u].y);
            } else {
                nx.x = fmaf(sdt, acc[u].x + kx, y0[u].x);
                nx.y = fmaf(sdt, acc[u].y + ky, y0[u].y);
                y0[u] = nx;
            }
            if (qi >= i) sts(own + dnext, nx);
            if (qi == i) dnew = nx.x;
            if (band_t && (unsigned)(qi - i - 1) < (unsigned)a.bw)
                sts(__float_as_int(m2f.w) + mir_lane, make_float2(nx.x, -nx.y));
            vprev = vcur;
            vcur = vnext;
        }
        const uint32_t ta = t0 + (uint32_t)(8 * j);
        if constexpr (!FINAL) tm_st4(ta + 4, acc[0], acc[1]);
        else tm_st8z(ta, y0[0], y0[1]);
    }
    publish_diag<FINAL, CLUSTER>(a, c, diag_t && (unsigned)qi < (unsigned)kR, cur, slot, s, q, dnew, b_id, snap_now,
                                 snap_row);
}

template <bool FINAL, bool PM1, bool CLUSTER>
__device__ __forceinline__ void tile_stage(const TileArgs &a, const TileCtx &c, const StageC &sc, long long b_id,
                                           bool snap_now, long long snap_row)
{
    int e = 0;   // row pairs of this warp done so far (tensor-memory column / 8)
    for (int it = 0; it < a.k_tiles; ++it) {
        const uint2 td = __ldg(&c.tiles[it]);
        if (td.x == 0xFFFFFFFFu) break;
        if (PM1 && (td.y & kFull)) {
            if (td.y & kRemote) tile_rows8<FINAL, CLUSTER, true>(a, c, sc, td, e, b_id, snap_now, snap_row);
            else tile_rows8<FINAL, CLUSTER, false>(a, c, sc, td, e, b_id, snap_now, snap_row);
            e += kR / 2;
        } else {
            tile_rows<FINAL, PM1, CLUSTER>(a, c, sc, td, e, b_id, snap_now, snap_row);
            e += (td_cnt(td.x) + 1) >> 1;
        }
    }
}

// Per-problem set-up of a CTA: shared-memory offsets of the problem's
// diagonal table, row table and stage buffers; both stage buffers zeroed
// (padding slots stay finite) and this rank's row table copied in.  Ends
// with a CTA barrier.
template <int WARPS>
__device__ __forceinline__ void tile_setup(const TileArgs &a, TileCtx &c, int warp)
{
    const int twoN = 2 * a.N;
    const int diag_bytes = 16 * ((4 * 2 * a.S * twoN + 15) / 16);
    c.diag_off = 64;
    c.rows_off = 64 + diag_bytes;
    c.buf0 = 64 + diag_bytes + a.rows_bytes;
    c.rb0 = a.row_begin[c.rank];
    c.rb1 = a.row_begin[c.rank + 1];
    c.tiles = a.tiles + ((size_t)c.rank * WARPS + warp) * a.k_tiles;
    for (int i = threadIdx.x; i < (2 * a.buf_bytes) / 16; i += blockDim.x)
        reinterpret_cast<float4 *>(tile_smem + c.buf0)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = threadIdx.x; i < (c.rb1 - c.rb0) * (int)(sizeof(RowEntry) / 16); i += blockDim.x)
        reinterpret_cast<uint4 *>(tile_smem + c.rows_off)[i] = __ldg(reinterpret_cast<const uint4 *>(a.rows + c.rb0) + i);
    __syncthreads();
}

// One batch of S samples: load rho(0), n_steps RK4 steps, write rho(T) back.
// Starts and ends at a barrier of the cluster (or CTA).
template <bool PM1, bool CLUSTER, int WARPS>
__device__ __forceinline__ void tile_batch(const TileArgs &a, const TileCtx &c, int warp, long long b_id)
{
    const int N = a.N, S = a.S, twoN = 2 * N, lane = c.lane;
    // ---- load rho(0): stored elements (upper part and mirror band) of own rows
    for (int slot = 0; slot < S; ++slot) {
        const long long m = b_id * S + slot;
        const int slot_off = slot * a.slot_bytes;
        for (int sr = c.rb0 + warp; sr < c.rb1; sr += WARPS) {
            const int s = sr / N, p = sr % N, lo = p > a.bw ? p - a.bw : 0;
            for (int k = lo + lane; k < N; k += 32) {
                float2 v = make_float2(0.f, 0.f);
                if (m < a.M) {
                    if (k >= p) {
                        v = a.rho[((m * 2 + s) * N + p) * (long long)N + k];
                    } else {
                        v = a.rho[((m * 2 + s) * N + k) * (long long)N + p];
                        v.y = -v.y;
                    }
                }
                if (k == p) {
                    v.y = 0.f;
                    if (a.snap && m < a.M) a.snap[m * twoN + s * N + p] = v.x;
                    const int di = slot * twoN + s * N + p;   // stage buffer 0
                    if constexpr (CLUSTER) {
                        const uint32_t da = c.diag_s + (uint32_t)(4 * di);
                        for (int r = 0; r < a.C; ++r) {
                            const uint32_t ra = map_rank(da, c.rank_base + (uint32_t)r);
                            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(ra), "f"(v.x) : "memory");
                        }
                    } else {
                        *reinterpret_cast<float *>(tile_smem + c.diag_off + 4 * di) = v.x;
                    }
                }
                const int off = c.buf0 + slot_off + elem_off(a.zoff[c.rank], s, p, k, a.qoff);
                *reinterpret_cast<float2 *>(tile_smem + off) = v;
            }
        }
    }
    // y0 of the computed elements into tensor memory, accumulators zeroed
    {
        int e = 0;
        for (int it = 0; it < a.k_tiles; ++it) {
            const uint2 td = __ldg(&c.tiles[it]);
            if (td.x == 0xFFFFFFFFu) break;
            const int p0 = td_p0(td.x), cnt = td_cnt(td.x), blk = td_blk(td.x), slot = td_slot(td.x);
            const int s = p0 >= N ? 1 : 0;
            const int q = lane < kW ? a.qoff + kW * blk + lane : kIdleQ;
            const long long m = b_id * S + slot;
            for (int i = 0; i < cnt; i += 2) {
                float2 v[2];
                for (int j = 0; j < 2; ++j) {
                    const int p = p0 - s * N + i + j;
                    v[j] = make_float2(0.f, 0.f);
                    if (i + j < cnt && q >= p && q < N && m < a.M) {
                        v[j] = a.rho[((m * 2 + s) * N + p) * (long long)N + q];
                        if (q == p) v[j].y = 0.f;
                    }
                }
                __syncwarp();
                tm_st8z(c.t_state + (uint32_t)(8 * (e + (i >> 1))), v[0], v[1]);
            }
            e += (cnt + 1) >> 1;
        }
    }
    tmem_wait_st();
    stage_sync<CLUSTER>();

    const float hdt = a.dt * 0.5f;
    for (long long step = 0; step < a.n_steps; ++step) {
        const bool snap_now = a.snap && ((step + 1) % a.out_every == 0);
        const long long snap_row = (step + 1) / a.out_every;
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {
            const StageC sc{k & 1, k == 0 ? 1.f : 2.f, k == 2 ? a.dt : hdt};
            tile_stage<false, PM1, CLUSTER>(a, c, sc, b_id, snap_now, snap_row);
            tmem_wait_st();
            stage_sync<CLUSTER>();
        }
        tile_stage<true, PM1, CLUSTER>(a, c, StageC{1, 0.f, 0.f}, b_id, snap_now, snap_row);
        tmem_wait_st();
        stage_sync<CLUSTER>();
    }

    // ---- write back rho(T) (full Hermitian matrix) from the y0 words
    {
        int e = 0;
        for (int it = 0; it < a.k_tiles; ++it) {
            const uint2 td = __ldg(&c.tiles[it]);
            if (td.x == 0xFFFFFFFFu) break;
            const int p0 = td_p0(td.x), cnt = td_cnt(td.x), blk = td_blk(td.x), slot = td_slot(td.x);
            const int s = p0 >= N ? 1 : 0;
            const int q = lane < kW ? a.qoff + kW * blk + lane : kIdleQ;
            const long long m = b_id * S + slot;
            for (int i = 0; i < cnt; i += 2) {
                uint32_t w[8];
                __syncwarp();
                tm_ld8(c.t_state + (uint32_t)(8 * (e + (i >> 1))), w);
                tm_wait8(w);
                for (int j = 0; j < 2 && i + j < cnt; ++j) {
                    const int p = p0 - s * N + i + j;
                    const float2 y = make_float2(__uint_as_float(w[2 * j]), __uint_as_float(w[2 * j + 1]));
                    if (q >= p && q < N && m < a.M) {
                        if (!(isfinite(y.x) && isfinite(y.y))) atomicCAS(a.status, 0, FTWA_ERR_NONFINITE);
                        a.rho[((m * 2 + s) * N + p) * (long long)N + q] = y;
                        if (p != q) a.rho[((m * 2 + s) * N + q) * (long long)N + p] = make_float2(y.x, -y.y);
                    }
                }
            }
            e += (cnt + 1) >> 1;
        }
    }
    __syncwarp();
    // the next batch overwrites the stage buffers that peers read until here
    stage_sync<CLUSTER>();
}

template <bool PM1, bool CLUSTER, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) tile_stepper(const __grid_constant__ TileArgs a)
{
    constexpr int WARPS = THREADS / 32;
    unsigned char *smem = tile_smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t cid = CLUSTER ? cluster_id_x() : blockIdx.x;
    const uint32_t ncl = CLUSTER ? n_clusters_x() : gridDim.x;

    // shared memory: header (64 B) | diagonals [2][S][2N] | row table | stage buffers 0, 1
    TileHeader *h = reinterpret_cast<TileHeader *>(smem);
    TileCtx c;
    c.smem_s = smem_addr(smem);
    c.diag_s = smem_addr(smem + 64);
    c.rank = (int)rank;
    c.rank_base = 0;
    c.lane = lane;
    c.prev_c = 0;
    c.next_c = 0;
    if constexpr (CLUSTER) {
        if (rank > 0) c.prev_c = map_rank(c.smem_s, rank - 1);
        if ((int)rank + 1 < a.C) c.next_c = map_rank(c.smem_s, rank + 1);
    }
    if (threadIdx.x == 0) {
        h->abort = 0;
        mbar_init(smem_addr(&h->dead_bar), 1u);
        fence_mbar_init_cluster();
    }
    tile_setup<WARPS>(a, c, warp);
    if (warp == 0) {
        tmem_alloc(smem_addr(&h->tmem_base), kTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if constexpr (CLUSTER) cluster_sync_hw();
    c.t_state = h->tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cols_per_warp(WARPS) * (warp >> 2));

    if (a.force_timeout) {
        // test hook: a bounded wait on a barrier that nothing arrives at; every
        // CTA gives up the same way and skips the integration
        if (threadIdx.x == 0 && !mbar_wait_bounded(smem_addr(&h->dead_bar), 0u, a.timeout_ns)) {
            h->abort = 1;
            atomicCAS(a.status, 0, FTWA_ERR_DEVICE_TIMEOUT);
        }
        __syncthreads();
    }

    const long long n_batches = (a.M + a.S - 1) / a.S;
    const bool run = h->abort == 0;
    for (long long b_id = cid; run && b_id < n_batches; b_id += ncl) tile_batch<PM1, CLUSTER, WARPS>(a, c, warp, b_id);

    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(h->tmem_base, kTmemCols);
    if constexpr (CLUSTER) cluster_sync_hw();
}

// Problems of a persistent batched launch (kernel parameter space).
constexpr int kMaxBatch = 24;
struct BatchArgs {
    int n_items, C;
    const int2 *items;   // [n_items]: (problem, batch of S samples), largest cost first
    int *counter;        // work-queue head, zeroed before every launch
    TileArgs prob[kMaxBatch];
};

// One persistent cluster-launched kernel over a queue of (problem, sample
// batch) work items of problems of different lattices and U: each cluster
// takes the next item (its rank 0 draws it and hands it to the cluster's
// CTAs), sets the problem up when it changes, and integrates the batch.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1) tile_batch_stepper(const __grid_constant__ BatchArgs B)
{
    constexpr int WARPS = THREADS / 32;
    unsigned char *smem = tile_smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    TileHeader *h = reinterpret_cast<TileHeader *>(smem);
    TileCtx c;
    c.smem_s = smem_addr(smem);
    c.diag_s = smem_addr(smem + 64);
    c.lane = lane;
    c.prev_c = rank > 0 ? map_rank(c.smem_s, rank - 1) : 0u;
    c.next_c = (int)rank + 1 < B.C ? map_rank(c.smem_s, rank + 1) : 0u;
    if (warp == 0) {
        tmem_alloc(smem_addr(&h->tmem_base), kTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    cluster_sync_hw();
    c.t_state = h->tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(cols_per_warp(WARPS) * (warp >> 2));

    int cur = -1;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int it = atomicAdd(B.counter, 1);
            const uint32_t ia = smem_addr(&h->item);
            for (int r = 0; r < B.C; ++r) {
                const uint32_t ra = map_rank(ia, (uint32_t)r);
                asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(ra), "r"(it) : "memory");
            }
        }
        stage_sync<true>();
        const int it = *reinterpret_cast<volatile int *>(&h->item);
        if (it >= B.n_items) break;
        const int2 w = __ldg(&B.items[it]);
        const TileArgs &a = B.prob[w.x];
        // a problem decomposed over a.C CTAs runs B.C / a.C batches of the
        // item side by side, one per group of a.C CTAs of the cluster
        const int groups = B.C / a.C;
        c.rank = (int)rank % a.C;
        c.rank_base = rank - (uint32_t)c.rank;
        const long long b_id = (long long)w.y * groups + (int)rank / a.C;
        if (w.x != cur) {
            tile_setup<WARPS>(a, c, warp);
            cur = w.x;
        }
        if (a.C == 1) {
            if (a.pm1) tile_batch<true, false, WARPS>(a, c, warp, b_id);
            else tile_batch<false, false, WARPS>(a, c, warp, b_id);
        } else {
            if (a.pm1) tile_batch<true, true, WARPS>(a, c, warp, b_id);
            else tile_batch<false, true, WARPS>(a, c, warp, b_id);
        }
    }

    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(h->tmem_base, kTmemCols);
    cluster_sync_hw();
}

// ---------------------------------------------------------------------------
// Host side: work decomposition (pure host code, also used by the layout check)
// ---------------------------------------------------------------------------
struct Nbr {
    int k[3];
    double t[3];
    int deg;
};

struct Layout {
    int N = 0, bw = 0, nblk = 0, qoff = 0, C = 1, S = 1, pm1 = 0;
    int slot_bytes = 0, buf_bytes = 0, smem_bytes = 0, k_tiles = 0, rows_bytes = 0;
    int row_begin[kMaxCluster + 1] = {0};
    int zoff[kMaxCluster][2][kMaxBlk] = {};
    int warps = 24;                              // warps per CTA
    std::vector<uint2> tiles;                    // [C][warps][k_tiles]
    std::vector<int4> koff;                      // [C][nblk][32]
    std::vector<float2> tq;                      // [nblk][32][3]
    std::vector<RowEntry> rows;                  // [2N]
    std::vector<RowPm1> rows_pm1;                // [2N], carried-row lattices: the table the kernel reads
    std::vector<int> rp_k;                       // [nblk][32][3] column read by each row-part slot
    std::vector<char> rp_real;                   // [nblk][32][3] the slot is a bond (else zero hopping)
    std::vector<int> slices;                     // per rank
};

static void neighbours(const Plan *p, std::vector<Nbr> &nb)
{
    const int N = p->N;
    nb.assign(N, Nbr{{0, 0, 0}, {0, 0, 0}, 0});
    for (size_t b = 0; b < p->t_bond.size(); ++b) {
        const int i = p->bonds[2 * b], j = p->bonds[2 * b + 1];
        nb[i].k[nb[i].deg] = j;
        nb[i].t[nb[i].deg++] = p->t_bond[b];
        nb[j].k[nb[j].deg] = i;
        nb[j].t[nb[j].deg++] = p->t_bond[b];
    }
}

// every site's neighbours among p - 1, p + 1 and at most one other site
static bool is_pm1(const std::vector<Nbr> &nb)
{
    const int N = (int)nb.size();
    for (int p = 0; p < N; ++p) {
        int far = 0;
        for (int n = 0; n < nb[p].deg; ++n)
            if (std::abs(nb[p].k[n] - p) != 1) ++far;
        if (far > 1) return false;
    }
    return true;
}

// rank of spin-row sr
static int owner(const Layout &L, int sr)
{
    int r = 0;
    while (r + 1 < L.C && sr >= L.row_begin[r + 1]) ++r;
    return r;
}

// Row-part slots of every column (depends on the lattice only; computed once
// per plan): the column read by each of a lane's three gathers and its hopping.
struct RowSlots {
    std::vector<int> k;         // [nblk][32][3]
    std::vector<char> real;     // [nblk][32][3]
    std::vector<float2> tq;     // [nblk][32][3]
};
static void row_part_slots(int N, int bw, const std::vector<Nbr> &nb, RowSlots &rs)
{
    // Each lane's neighbours may sit in any of the three slots (a slot is one
    // warp-wide gather), and a missing neighbour reads a stored decoy column
    // with zero hopping.  Per 16-lane half-warp the assignment and the decoys
    // are searched so that each gather touches as few words per shared-memory
    // bank pair as possible (the bank pair of column k in any row is
    // lane(k) mod 16 in this layout; lanes reading the same column share a
    // word).  The idle lane 31 repeats lane 30's reads.
    const int nblk = (N + kW - 1) / kW, qoff = N - kW * nblk;
    rs.k.assign((size_t)nblk * 32 * 3, 0);
    rs.real.assign((size_t)nblk * 32 * 3, 0);
    rs.tq.assign((size_t)nblk * 32 * 3, make_float2(0.f, 0.f));
    auto bank = [&](int k) { return lane_of(k, qoff) % 16; };
    struct Ent {
        int k;
        bool real;
        float t;
    };
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int b = 0; b < nblk; ++b)
        for (int h = 0; h < 2; ++h) {
            const int l0 = 16 * h, l1 = std::min(16 * h + 16, kW), nl = l1 - l0;
            Ent ent0[16][3];
            int qv[16];
            for (int j = 0; j < nl; ++j) {
                const int q = qoff + kW * b + l0 + j;
                qv[j] = q;
                const int qq = q < 0 ? 0 : q;
                for (int n = 0; n < 3; ++n) ent0[j][n] = Ent{qq, false, 0.f};
                if (q < 0) continue;
                for (int n = 0; n < nb[q].deg; ++n) ent0[j][n] = Ent{nb[q].k[n], true, (float)nb[q].t[n]};
            }
            Ent ent[16][3];
            int perm[16][3];   // slot n holds ent[j][perm[j][n]]
            // distinct words of slot n (lane `skip` left out), and their bank-pair counts
            auto slot_words = [&](int n, int skip, int *cols, int &nc, int *pc) {
                nc = 0;
                for (int x = 0; x < 16; ++x) pc[x] = 0;
                for (int j = 0; j < nl; ++j) {
                    if (j == skip) continue;
                    const int k = ent[j][perm[j][n]].k;
                    bool seen = false;
                    for (int x = 0; x < nc && !seen; ++x) seen = cols[x] == k;
                    if (seen) continue;
                    cols[nc++] = k;
                    pc[bank(k)]++;
                }
            };
            auto cost = [&]() {
                long long c = 0;
                int cols[16], nc, pc[16];
                for (int n = 0; n < 3; ++n) {
                    slot_words(n, -1, cols, nc, pc);
                    int mx = 0, sq = 0;
                    for (int x = 0; x < 16; ++x) {
                        mx = std::max(mx, pc[x]);
                        sq += pc[x] * pc[x];
                    }
                    c += 1000 * mx + sq;
                }
                return c;
            };
            // decoys of lane j: a column another lane of the slot already reads,
            // else a stored column on the least used bank pair
            auto place_decoys = [&](int j) {
                int cols[16], nc, pc[16];
                for (int n = 0; n < 3; ++n) {
                    Ent &e = ent[j][perm[j][n]];
                    if (e.real) continue;
                    slot_words(n, j, cols, nc, pc);
                    const int q = qv[j];
                    int best = q, best_c = 1 << 30;
                    for (int d = 0; d <= bw; ++d)
                        for (int sg = 1; sg >= -1; sg -= 2) {
                            const int k = q + sg * d;
                            if (k < 0 || k >= N || k < q - bw) continue;
                            bool shared = false;
                            for (int x = 0; x < nc && !shared; ++x) shared = cols[x] == k;
                            const int c = shared ? 0 : 1 + 4 * pc[bank(k)];
                            if (c < best_c) {
                                best_c = c;
                                best = k;
                            }
                        }
                    e.k = best;
                }
            };
            // starting points: the neighbour order, the pattern where lanes j and
            // j + 2 read their common neighbour column in one slot, and
            // pseudo-random orders; a local search (one lane's order at a time)
            // from each, the best kept
            Ent best_ent[16][3];
            int best_perm[16][3];
            long long best_all = -1;
            uint32_t rng = 0x9E3779B9u ^ (uint32_t)(b * 2 + h);
            for (int start = 0; start < 16 && best_all != 3000 + 3 * nl; ++start) {
                for (int j = 0; j < nl; ++j) {
                    for (int n = 0; n < 3; ++n) ent[j][n] = ent0[j][n];
                    int x = 0;
                    if (start == 1 && qv[j] >= 0) {
                        int ip = -1, im = -1;
                        for (int n = 0; n < 3; ++n) {
                            if (ent[j][n].real && ent[j][n].k == qv[j] + 1) ip = n;
                            if (ent[j][n].real && ent[j][n].k == qv[j] - 1) im = n;
                        }
                        if (ip >= 0 && im >= 0) {
                            const int first = (j & 3) < 2 ? ip : im, second = (j & 3) < 2 ? im : ip;
                            for (int y = 0; y < 6; ++y)
                                if (perms[y][0] == first && perms[y][1] == second) x = y;
                        }
                    } else if (start > 1 && qv[j] >= 0) {
                        rng = rng * 1664525u + 1013904223u;
                        x = (int)((rng >> 16) % 6);
                    }
                    for (int n = 0; n < 3; ++n) perm[j][n] = perms[x][n];
                }
                for (int j = 0; j < nl; ++j)
                    if (qv[j] >= 0) place_decoys(j);
                long long cur = cost();
                for (int pass = 0; pass < 8; ++pass) {
                    bool improved = false;
                    for (int j = 0; j < nl; ++j) {
                        if (qv[j] < 0) continue;
                        Ent keep_e[3], bst_e[3];
                        int bst_p[3];
                        for (int n = 0; n < 3; ++n) {
                            keep_e[n] = bst_e[n] = ent[j][n];
                            bst_p[n] = perm[j][n];
                        }
                        long long bst = cur;
                        for (int y = 0; y < 6; ++y) {
                            for (int n = 0; n < 3; ++n) {
                                ent[j][n] = keep_e[n];
                                perm[j][n] = perms[y][n];
                            }
                            place_decoys(j);
                            const long long c = cost();
                            if (c < bst) {
                                bst = c;
                                for (int n = 0; n < 3; ++n) {
                                    bst_e[n] = ent[j][n];
                                    bst_p[n] = perm[j][n];
                                }
                            }
                        }
                        for (int n = 0; n < 3; ++n) {
                            ent[j][n] = bst_e[n];
                            perm[j][n] = bst_p[n];
                        }
                        if (bst < cur) {
                            cur = bst;
                            improved = true;
                        }
                    }
                    if (!improved) break;
                }
                if (best_all < 0 || cur < best_all) {
                    best_all = cur;
                    for (int j = 0; j < nl; ++j)
                        for (int n = 0; n < 3; ++n) {
                            best_ent[j][n] = ent[j][n];
                            best_perm[j][n] = perm[j][n];
                        }
                }
            }
            for (int j = 0; j < nl; ++j)
                for (int n = 0; n < 3; ++n) {
                    const Ent &e = best_ent[j][best_perm[j][n]];
                    const size_t ix = (size_t)(b * 32 + l0 + j) * 3 + n;
                    rs.k[ix] = e.k;
                    rs.real[ix] = e.real ? 1 : 0;
                    rs.tq[ix] = e.real ? make_float2(e.t, e.t) : make_float2(0.f, 0.f);
                }
        }
}

// The plan's row-part slots: searched on first use, then kept in the plan.
static void plan_row_slots(Plan *p, const std::vector<Nbr> &nb, RowSlots &rs)
{
    if (p->tile_rp_k.empty()) {
        row_part_slots(p->N, p->bandwidth, nb, rs);
        p->tile_rp_k = rs.k;
        p->tile_rp_real = rs.real;
        p->tile_rp_t.resize(2 * rs.tq.size());
        for (size_t i = 0; i < rs.tq.size(); ++i) {
            p->tile_rp_t[2 * i] = rs.tq[i].x;
            p->tile_rp_t[2 * i + 1] = rs.tq[i].y;
        }
        return;
    }
    rs.k = p->tile_rp_k;
    rs.real = p->tile_rp_real;
    rs.tq.resize(p->tile_rp_t.size() / 2);
    for (size_t i = 0; i < rs.tq.size(); ++i) rs.tq[i] = make_float2(p->tile_rp_t[2 * i], p->tile_rp_t[2 * i + 1]);
}

// Build the decomposition for C CTAs per sample and S slots (C == 1 only).
// Returns false when it does not fit (shared memory, tensor memory, ranks
// narrower than the bandwidth).
static bool build_layout(const Plan *p, const std::vector<Nbr> &nb, const RowSlots &rs, bool pm1, int C, int S,
                         int warps, Layout &L)
{
    const int N = p->N, bw = p->bandwidth;
    L = Layout();
    L.warps = warps;
    const int kWarpsT = warps;
    L.N = N;
    L.bw = bw;
    L.nblk = (N + kW - 1) / kW;
    L.qoff = N - kW * L.nblk;
    L.C = C;
    L.S = S;
    L.pm1 = pm1 ? 1 : 0;
    const int nblk = L.nblk, qoff = L.qoff;
    auto lastcol = [&](int b) { return qoff + kW * b + kW - 1; };
    auto cslices = [&](int p_) { return nblk - blk_of(p_, qoff); };
    if (C > kMaxCluster || (C > 1 && (C & 1))) return false;
    // ---- ranks: C == 1 both spins; C >= 2 each spin split in C/2 ranks, balanced by computed slices
    if (C == 1) {
        L.row_begin[0] = 0;
        L.row_begin[1] = 2 * N;
    } else {
        const int per = C / 2;
        std::vector<int> cut(per + 1, 0);
        double tot = 0;
        for (int x = 0; x < N; ++x) tot += cslices(x);
        int x = 0;
        double acc = 0;
        for (int r = 1; r < per; ++r) {
            const double target = tot * r / per;
            while (x < N && acc + 0.5 * cslices(x) < target) acc += cslices(x++);
            cut[r] = x;
        }
        cut[per] = N;
        for (int s = 0; s < 2; ++s)
            for (int r = 0; r < per; ++r) L.row_begin[s * per + r] = s * N + cut[r];
        L.row_begin[C] = 2 * N;
        for (int r = 0; r < C; ++r) {
            const int rows = L.row_begin[r + 1] - L.row_begin[r];
            if (rows < 1) return false;
            // column-part and mirror partners are at most bw rows away: they must
            // lie in this rank or an adjacent rank of the same spin
            if (per > 1 && rows < bw) return false;
        }
    }
    // ---- regions: per rank, spin, block: rows [P0, min(P1, lastcol + bw + 1))
    int slot_bytes = 0, max_rows = 0;
    for (int r = 0; r < C; ++r) {
        int off = 0;
        max_rows = std::max(max_rows, L.row_begin[r + 1] - L.row_begin[r]);
        for (int s = 0; s < 2; ++s) {
            const int P0 = std::max(L.row_begin[r], s * N) - s * N;
            const int P1 = std::min(L.row_begin[r + 1], s * N + N) - s * N;
            if (P1 <= P0) continue;
            for (int b = 0; b < nblk; ++b) {
                const int hi = std::max(P0, std::min(P1, lastcol(b) + bw + 1));
                const int rows = hi - P0;
                off = (off + 127) / 128 * 128;   // every region on a 128-byte boundary (bank pattern)
                L.zoff[r][s][b] = off - P0 * kRowBytes;
                off += rows * kRowBytes;
            }
        }
        slot_bytes = std::max(slot_bytes, off);
    }
    // slots and the stage buffers on 128-byte boundaries too: the row table is
    // padded so that the buffers start on one
    L.slot_bytes = (slot_bytes + 127) / 128 * 128;
    L.buf_bytes = S * L.slot_bytes;
    const int diag_bytes = 16 * ((4 * 2 * S * 2 * N + 15) / 16);
    L.rows_bytes = max_rows * (int)sizeof(RowEntry);
    L.rows_bytes += (128 - (64 + diag_bytes + L.rows_bytes) % 128) % 128;
    L.smem_bytes = 64 + diag_bytes + L.rows_bytes + 2 * L.buf_bytes;
    if (L.smem_bytes > 227 * 1024) return false;

    // ---- column-part table (per spin-row, from the owner's point of view)
    L.rows.assign((size_t)2 * N, RowEntry{});
    for (int sr = 0; sr < 2 * N; ++sr) {
        const int s = sr / N, pp = sr % N, r = owner(L, sr);
        RowEntry e{};
        int slot_k[3] = {pp, pp, pp};      // empty slot: the own row, zero hopping
        double slot_t[3] = {0.0, 0.0, 0.0};
        if (pm1) {
            // slots: p - 1, p + 1, the far neighbour
            for (int n = 0; n < nb[pp].deg; ++n) {
                const int k = nb[pp].k[n];
                const int sl = k == pp - 1 ? 0 : (k == pp + 1 ? 1 : 2);
                slot_k[sl] = k;
                slot_t[sl] = nb[pp].t[n];
            }
        } else {
            for (int n = 0; n < nb[pp].deg; ++n) {
                slot_k[n] = nb[pp].k[n];
                slot_t[n] = nb[pp].t[n];
            }
        }
        for (int n = 0; n < 3; ++n) {
            e.mt[n] = -(float)slot_t[n];
            if (pm1 && n < 2) continue;          // carried rows p -+ 1
            const int k = slot_k[n];
            const int ksr = s * N + k;
            const bool remote = ksr < L.row_begin[r] || ksr >= L.row_begin[r + 1];
            if (remote) {
                const int o = owner(L, ksr);
                if (std::abs(o - r) != 1 || o / std::max(C / 2, 1) != r / std::max(C / 2, 1)) return false;
                e.flags |= 1u << n;
                if (o == r + 1) e.flags |= 1u << (3 + n);
                e.dcol[n] = kRowBytes * k;
            } else {
                e.dcol[n] = kRowBytes * (k - pp);
            }
        }
        e.mir = L.zoff[r][s][blk_of(pp, qoff)] + 8 * lane_of(pp, qoff);
        L.rows[sr] = e;
    }
    if (pm1) {
        L.rows_pm1.assign((size_t)2 * N, RowPm1{});
        for (int sr = 0; sr < 2 * N; ++sr) {
            const RowEntry &e = L.rows[sr];
            RowPm1 &f = L.rows_pm1[sr];
            f.m0[0] = f.m0[1] = e.mt[0];
            f.m1[0] = f.m1[1] = e.mt[1];
            f.m2[0] = f.m2[1] = e.mt[2];
            f.far = e.dcol[2];
            if (e.flags & 4u) f.far |= 1 | ((e.flags & 32u) ? 2 : 0);
            f.mir = e.mir;
        }
    }
    L.rp_k = rs.k;
    L.rp_real = rs.real;
    L.tq = rs.tq;
    L.koff.assign((size_t)C * nblk * 32, int4{0, 0, 0, 0});
    for (int r = 0; r < C; ++r) {
        const int s = L.row_begin[r] >= N ? 1 : 0;
        for (int b = 0; b < nblk; ++b)
            for (int ln = 0; ln < 32; ++ln) {
                int o[3];
                const int lr = std::min(ln, kW - 1);   // the idle lane repeats lane 30's reads
                for (int n = 0; n < 3; ++n) {
                    const int k = L.rp_k[(size_t)(b * 32 + lr) * 3 + n];
                    o[n] = L.zoff[r][s][blk_of(k, qoff)] - L.zoff[r][s][b] + 8 * (lane_of(k, qoff) - lr);
                }
                L.koff[((size_t)r * nblk + b) * 32 + ln] = int4{o[0], o[1], o[2], 0};
            }
    }
    if (C == 1 && N > 0) {
        // both spins share one table: their regions have the same sizes
        for (int b = 0; b < nblk; ++b)
            if (L.zoff[0][1][b] - L.zoff[0][1][0] != L.zoff[0][0][b] - L.zoff[0][0][0]) return false;
    }

    // ---- tiles, assigned to warps longest first under the tensor-memory cap
    const int pairs_cap = cols_per_warp(warps) / 8;
    std::vector<uint2> all_tiles;
    int kt = 1;
    std::vector<std::vector<uint2>> per_rank_warp((size_t)C * kWarpsT);
    L.slices.assign(C, 0);
    for (int r = 0; r < C; ++r) {
        std::vector<std::pair<int, uint2>> tl;
        for (int slot = 0; slot < S; ++slot)
            for (int s = 0; s < 2; ++s) {
                const int P0 = std::max(L.row_begin[r], s * N) - s * N;
                const int P1 = std::min(L.row_begin[r + 1], s * N + N) - s * N;
                if (P1 <= P0) continue;
                for (int b = 0; b < nblk; ++b) {
                    const int last = std::min(P1, lastcol(b) + 1);
                    for (int x = P0; x < last;) {
                        const int cnt = std::min(kR, last - x);
                        uint2 td;
                        td.x = td_make(s * N + x, cnt, b, slot);
                        uint32_t f = 0;
                        const int c0 = qoff + kW * b;
                        for (int i = 0; i < cnt; ++i) {
                            const int pp = x + i;
                            if (blk_of(pp, qoff) == b) f |= kDiag;
                            if (pp + bw >= c0 && pp < lastcol(b)) f |= kBand;
                            if (L.rows[s * N + pp].flags & 7u) f |= kRemote;
                            if (pp + bw >= c0 && pp < lastcol(b) && s * N + pp + bw >= L.row_begin[r + 1]) f |= kRemoteMir;
                        }
                        if (pm1) {
                            const int prev = x - 1, next = x + cnt;
                            uint32_t pk = 0, nk = 0;
                            if (prev < P0) pk = prev < 0 ? 1u : 2u;
                            if (next >= P1) nk = next >= N ? 1u : 2u;
                            if (pk == 2 && r == 0) return false;
                            if (nk == 2 && r + 1 >= C) return false;
                            f |= pk << kPrevShift;
                            f |= nk << kNextShift;
                        }
                        if (pm1 && cnt == kR && !(f & kRemoteMir)) {
                            // remote far slots of the tile: all in one neighbour rank
                            bool prev = false, next = false;
                            for (int i = 0; i < cnt; ++i) {
                                const uint32_t fl = L.rows[s * N + x + i].flags;
                                if (fl & 4u) ((fl & 32u) ? next : prev) = true;
                            }
                            if (!(prev && next)) f |= kFull | (next ? kFarNext : 0u);
                        }
                        td.y = f;
                        // cost weight (per row, x100): unrolled tiles, with remote far slots, general path
                        const int wgt = (f & kFull) ? ((f & kRemote) ? 110 : 100) : 150;
                        tl.push_back({cnt * wgt, td});
                        L.slices[r] += cnt;
                        x += cnt;
                    }
                }
            }
        std::stable_sort(tl.begin(), tl.end(), [](const auto &u, const auto &v) { return u.first > v.first; });
        std::vector<int> load(kWarpsT, 0), pairs(kWarpsT, 0);
        for (const auto &t : tl) {
            int w = -1;
            const int tc = td_cnt(t.second.x);
            for (int x = 0; x < kWarpsT; ++x)
                if (pairs[x] + (tc + 1) / 2 <= pairs_cap && (w < 0 || load[x] < load[w])) w = x;
            if (w < 0) return false;
            load[w] += t.first;
            pairs[w] += (tc + 1) / 2;
            per_rank_warp[(size_t)r * kWarpsT + w].push_back(t.second);
        }
        for (int x = 0; x < kWarpsT; ++x) kt = std::max<int>(kt, (int)per_rank_warp[(size_t)r * kWarpsT + x].size());
    }
    L.k_tiles = kt;
    L.tiles.assign((size_t)C * kWarpsT * kt, uint2{0xFFFFFFFFu, 0u});
    for (size_t rw = 0; rw < per_rank_warp.size(); ++rw)
        for (size_t i = 0; i < per_rank_warp[rw].size(); ++i) L.tiles[rw * kt + i] = per_rank_warp[rw][i];
    return true;
}

// Simulate every shared-memory address the kernel forms for one sample slot
// and check it: reads of active lanes hit the intended element (or the zero
// row for empty slots), every read stays inside the buffer of the rank it
// addresses, every computed element is written exactly once per stage and
// every mirror-band entry exactly once.  Returns the number of violations.
static long long check_layout(const Layout &L, const std::vector<Nbr> &nb, char *msg, int msg_len)
{
    const int N = L.N, nblk = L.nblk, qoff = L.qoff, C = L.C;
    long long bad = 0;
    auto note = [&](const char *what, int r, int sr, int q) {
        if (bad++ == 0 && msg) snprintf(msg, (size_t)msg_len, "%s (rank %d, row %d, column %d)", what, r, sr, q);
    };
    // logical element of every stored byte offset, per rank: key = s*N*N + p*N + q
    std::vector<std::vector<int>> who(C, std::vector<int>((size_t)L.slot_bytes / 8 + 1, -1));
    for (int r = 0; r < C; ++r)
        for (int sr = L.row_begin[r]; sr < L.row_begin[r + 1]; ++sr) {
            const int s = sr / N, p = sr % N, lo = p > L.bw ? p - L.bw : 0;
            for (int q = lo; q < N; ++q) {
                const int off = elem_off(L.zoff[r], s, p, q, qoff);
                if (off < 0 || off + 8 > L.slot_bytes || (off & 7)) {
                    note("stored element outside the slot", r, sr, q);
                    continue;
                }
                if (who[r][off / 8] != -1) note("two elements share a slot", r, sr, q);
                who[r][off / 8] = (s * N + p) * N + q;
            }
        }
    auto read_ok = [&](int r, int off, int want, bool active, int sr, int q, const char *what) {
        if (off < 0 || off + 8 > L.slot_bytes || (off & 7)) {
            note(what, r, sr, q);
            return;
        }
        if (!active) return;
        if (who[r][off / 8] != want) note(what, r, sr, q);
    };
    std::vector<int> writes((size_t)2 * N * N, 0), mwrites((size_t)2 * N * N, 0), dwrites((size_t)2 * N, 0);
    for (int r = 0; r < C; ++r)
        for (int w = 0; w < L.warps; ++w)
            for (int it = 0; it < L.k_tiles; ++it) {
                const uint2 td = L.tiles[((size_t)r * L.warps + w) * L.k_tiles + it];
                if (td.x == 0xFFFFFFFFu) break;
                const int p0 = td_p0(td.x), cnt = td_cnt(td.x), b = td_blk(td.x), slot = td_slot(td.x);
                if (slot != 0) continue;
                const int s = p0 >= N ? 1 : 0, pp0 = p0 - s * N;
                // diagonal-table writes (once per row of a tile holding the row's diagonal)
                for (int i = 0; i < cnt; ++i) {
                    const int c0 = qoff + kW * b, p = pp0 + i;
                    if ((td.y & kDiag) && (unsigned)(p - c0) < (unsigned)kW) dwrites[(size_t)s * N + p]++;
                }
                for (int ln = 0; ln < 32; ++ln) {
                    // the idle lane 31 reads lane 30's addresses and writes nothing
                    const int lr = std::min(ln, kW - 1);
                    const int q = ln < kW ? qoff + kW * b + ln : kIdleQ;
                    const int4 ko = L.koff[((size_t)r * nblk + b) * 32 + ln];
                    const int own0 = L.zoff[r][s][b] + kRowBytes * pp0 + 8 * lr;
                    for (int i = 0; i < cnt; ++i) {
                        const int p = pp0 + i, sr = s * N + p;
                        const bool act = q >= p && q < N && q >= 0;
                        const int own = own0 + kRowBytes * i;
                        read_ok(r, own, (s * N + p) * N + q, act, sr, q, "own read");
                        const int kk[3] = {ko.x, ko.y, ko.z};
                        for (int n = 0; n < 3; ++n) {
                            const size_t ix = (size_t)(b * 32 + ln) * 3 + n;
                            const bool real = L.rp_real[ix] != 0;
                            const int k = L.rp_k[ix];
                            // a decoy of an active lane must still read a stored element of row p
                            const bool stored = k >= (p > L.bw ? p - L.bw : 0);
                            read_ok(r, own + kk[n], (s * N + p) * N + k, act && (real || stored), sr, q,
                                    real ? "row-part read" : "row-part decoy read");
                            if (act && !real && !stored) note("row-part decoy outside the stored band", r, sr, q);
                        }
                        const RowEntry &e = L.rows[sr];
                        for (int n = 0; n < 3; ++n) {
                            if (L.pm1) {
                                const RowPm1 &f = L.rows_pm1[sr];
                                const float *m = n == 0 ? f.m0 : (n == 1 ? f.m1 : f.m2);
                                if (m[0] != e.mt[n] || m[1] != e.mt[n]) note("row table hopping pair", r, sr, q);
                            }
                            if (L.pm1 && n == 2) {
                                // the far slot as the kernel decodes it
                                const int far = L.rows_pm1[sr].far;
                                if (L.rows_pm1[sr].mir != e.mir) note("row table mirror offset", r, sr, q);
                                if ((td.y & kFull) && (far & 1) && (((far & 2) != 0) != ((td.y & kFarNext) != 0)))
                                    note("remote far slot outside the fast tile's far rank", r, sr, q);
                                if (far & 1) {
                                    const int o = (far & 2) ? r + 1 : r - 1;
                                    const int k = (far & ~3) / kRowBytes;
                                    if (o < 0 || o >= C) {
                                        note("far slot in a rank outside the cluster", r, sr, q);
                                        continue;
                                    }
                                    read_ok(o, L.zoff[o][s][b] + (far & ~3) + 8 * lr, (s * N + k) * N + q, act, sr, q,
                                            "far column-part read (remote)");
                                } else {
                                    if (far & 3) note("far slot offset not row aligned", r, sr, q);
                                    const int k = p + far / kRowBytes;
                                    read_ok(r, own + far, (s * N + k) * N + q, act, sr, q, "far column-part read");
                                }
                                continue;
                            }
                            if (L.pm1 && n < 2) {
                                // carried rows p -+ 1: from the tile, or the boundary rows
                                const int k = n == 0 ? p - 1 : p + 1;
                                const bool in_tile = n == 0 ? i > 0 : i + 1 < cnt;
                                if (in_tile || e.mt[n] == 0.f) continue;
                                const uint32_t kind = (td.y >> (n == 0 ? kPrevShift : kNextShift)) & 3;
                                if (kind == 2) {
                                    const int o = n == 0 ? r - 1 : r + 1;
                                    read_ok(o, L.zoff[o][s][b] + kRowBytes * k + 8 * lr, (s * N + k) * N + q, act, sr, q,
                                            "boundary-row read (remote)");
                                } else if (kind == 0) {
                                    read_ok(r, own + (n == 0 ? -kRowBytes : kRowBytes), (s * N + k) * N + q, act, sr,
                                            q, "boundary-row read");
                                } else {
                                    note("absent boundary row with a nonzero hopping", r, sr, q);
                                }
                                continue;
                            }
                            if (e.flags & (1u << n)) {
                                const int o = (e.flags >> (3 + n)) & 1u ? r + 1 : r - 1;
                                const int k = e.dcol[n] / kRowBytes;
                                read_ok(o, L.zoff[o][s][b] + e.dcol[n] + 8 * lr, (s * N + k) * N + q, act, sr, q,
                                        "column-part read (remote)");
                            } else {
                                const int k = p + e.dcol[n] / kRowBytes;
                                read_ok(r, own + e.dcol[n], (s * N + k) * N + q, act, sr, q, "column-part read");
                            }
                        }
                        if (act) {
                            writes[(size_t)(s * N + p) * N + q]++;
                            if (q > p && q - p <= L.bw) {
                                const int qsr = s * N + q;
                                const int o = qsr < L.row_begin[r + 1] ? r : r + 1;
                                const int bp = blk_of(p, qoff);
                                const int mir_next = o < C ? e.mir - L.zoff[r][s][bp] + L.zoff[o][s][bp] : 0;
                                const int off = (o == r ? e.mir : mir_next) + kRowBytes * q;
                                if (o >= C) {
                                    note("mirror row beyond the last rank", r, sr, q);
                                } else if (o != r && !(td.y & kRemoteMir)) {
                                    note("mirror row in the next rank in a tile without kRemoteMir", r, sr, q);
                                } else {
                                    read_ok(o, off, (s * N + q) * N + p, true, sr, q, "mirror store");
                                    mwrites[(size_t)(s * N + q) * N + p]++;
                                }
                            }
                        }
                    }
                }
            }
    for (int sr = 0; sr < 2 * N; ++sr)
        if (dwrites[sr] != 1) note("diagonal not published exactly once", 0, sr, sr % N);
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q) {
                const size_t k = (size_t)(s * N + p) * N + q;
                if (q >= p && writes[k] != 1) note("computed element not written exactly once", 0, s * N + p, q);
                if (q < p && q >= p - L.bw && mwrites[k] != 1) note("mirror entry not written exactly once", 0, s * N + p, q);
                if ((q < p && writes[k]) || (q >= p && mwrites[k])) note("write outside its triangle", 0, s * N + p, q);
            }
    return bad;
}

// Choose C (1, 2, 4, 8) and S: the smallest cluster that fits, with as many
// slots as useful for C == 1.
// C_force / warps_force (0: the plan's overrides or defaults); multi_slot:
// several samples per cluster also for C > 1 (batched launches).
static bool choose_layout(const Plan *p, int64_t M, const std::vector<Nbr> &nb, const RowSlots &rs, bool pm1,
                          Layout &out,
                          int C_force = 0, int warps_force = 0, bool multi_slot = false)
{
    const int sm = p->sm_count > 0 ? p->sm_count : 1;
    const int warps = warps_force ? warps_force : (p->threads_override == 768 ? 24 : 16);
    for (int C = 1; C <= kMaxCluster; C *= 2) {
        if (C_force && C != C_force) continue;
        if (!C_force && p->cluster_override && C != p->cluster_override) continue;
        int want = 1;
        if (C == 1 || multi_slot)
            want = (int)std::max<long long>(1, std::min<long long>((M + sm / C - 1) / std::max(1, sm / C), 255));
        Layout best;
        bool ok = false;
        for (int S = 1; S <= want; ++S) {
            Layout L;
            if (!build_layout(p, nb, rs, pm1, C, S, warps, L)) break;
            best = L;
            ok = true;
        }
        if (ok) {
            out = best;
            return true;
        }
    }
    return false;
}

// Tables of a layout in one device-ready byte image: rows | tiles | koff | tq
// (16-byte aligned parts); offsets returned for the argument pointers.
struct TablePack {
    std::vector<unsigned char> bytes;
    size_t o_tiles = 0, o_koff = 0, o_tq = 0;
};
static void pack_tables(const Layout &L, TablePack &t)
{
    const size_t b_rows = L.rows.size() * sizeof(RowEntry);   // RowPm1 entries have the same size
    const size_t b_tiles = ((L.tiles.size() * sizeof(uint2) + 15) / 16) * 16;
    const size_t b_koff = L.koff.size() * sizeof(int4);
    const size_t b_tq = ((L.tq.size() * sizeof(float2) + 15) / 16) * 16;
    t.bytes.assign(b_rows + b_tiles + b_koff + b_tq, 0);
    t.o_tiles = b_rows;
    t.o_koff = b_rows + b_tiles;
    t.o_tq = b_rows + b_tiles + b_koff;
    if (L.pm1) std::memcpy(t.bytes.data(), L.rows_pm1.data(), b_rows);
    else std::memcpy(t.bytes.data(), L.rows.data(), b_rows);
    std::memcpy(t.bytes.data() + t.o_tiles, L.tiles.data(), L.tiles.size() * sizeof(uint2));
    std::memcpy(t.bytes.data() + t.o_koff, L.koff.data(), b_koff);
    std::memcpy(t.bytes.data() + t.o_tq, L.tq.data(), L.tq.size() * sizeof(float2));
}

// Kernel arguments of a layout whose tables are at device address `base`.
static void fill_args(const Plan *p, const Layout &L, const TablePack &t, const unsigned char *base, TileArgs &a)
{
    std::memset(&a, 0, sizeof(a));
    a.N = L.N;
    a.C = L.C;
    a.S = L.S;
    a.nblk = L.nblk;
    a.qoff = L.qoff;
    a.bw = L.bw;
    a.warps = L.warps;
    a.pm1 = L.pm1;
    a.slot_bytes = L.slot_bytes;
    a.buf_bytes = L.buf_bytes;
    a.k_tiles = L.k_tiles;
    a.U = (float)p->U;
    a.dt = (float)p->dt;
    a.out_every = p->out_every;
    a.status = p->d_status;
    a.timeout_ns = p->timeout_ns;
    a.force_timeout = p->force_timeout;
    for (int i = 0; i <= kMaxCluster; ++i) a.row_begin[i] = L.row_begin[std::min(i, L.C)];
    std::memcpy(a.zoff, L.zoff, sizeof(a.zoff));
    a.rows = reinterpret_cast<const RowEntry *>(base);
    a.rows_bytes = L.rows_bytes;
    a.tiles = reinterpret_cast<const uint2 *>(base + t.o_tiles);
    a.koff = reinterpret_cast<const int4 *>(base + t.o_koff);
    a.tq = reinterpret_cast<const float2 *>(base + t.o_tq);
}

}  // namespace tile

// FP32 plans with the on-site U (no drive or long-range field): the tiled
// stepper, when a shape fits.
bool tile_supported(const Plan *p)
{
    return p->precision == FTWA_FP32 && !p->drive && !p->longrange && !p->hop_drive && p->N <= FTWA_MAX_SITES &&
           p->N >= 2;
}

int launch_tile(Plan *p, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s)
{
    using namespace tile;
    if (!tile_supported(p)) return FTWA_ERR_UNSUPPORTED;
    std::vector<Nbr> nb;
    neighbours(p, nb);
    const bool pm1 = is_pm1(nb);
    Layout L;
    RowSlots rs;
    plan_row_slots(p, nb, rs);
    if (!choose_layout(p, M, nb, rs, pm1, L)) return FTWA_ERR_UNSUPPORTED;
    const int sm = p->sm_count > 0 ? p->sm_count : 1;
    const long long batches = (M + L.S - 1) / L.S;
    int grid = (int)std::min<long long>(std::max<long long>(batches, 1), std::max(1, sm / L.C)) * L.C;
    void (*kern)(TileArgs);
    if (L.warps == 16)
        kern = L.C > 1 ? (pm1 ? tile_stepper<true, true, 512> : tile_stepper<false, true, 512>)
                       : (pm1 ? tile_stepper<true, false, 512> : tile_stepper<false, false, 512>);
    else
        kern = L.C > 1 ? (pm1 ? tile_stepper<true, true, 768> : tile_stepper<false, true, 768>)
                       : (pm1 ? tile_stepper<true, false, 768> : tile_stepper<false, false, 768>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.smem_bytes);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(32 * L.warps, 1, 1);
    cfg.dynamicSmemBytes = L.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = L.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = L.C > 1 ? 1 : 0;
    if (L.C > 1) {
        int n_clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&n_clusters, kern, &cfg);
        if (e != cudaSuccess) return set_cuda_error(e);
        if (n_clusters < 1) return FTWA_ERR_UNSUPPORTED;
        grid = std::min(grid, n_clusters * L.C);
        cfg.gridDim = dim3(grid, 1, 1);
    }
    // tables in one plan-owned device buffer, uploaded when they change (never
    // during stream capture: batch creation prepares every plan first)
    TablePack tp;
    pack_tables(L, tp);
    const size_t bytes = tp.bytes.size();
    if (p->tile_bytes < bytes) {
        cudaFree(p->d_tile);
        p->d_tile = nullptr;
        p->tile_bytes = 0;
        e = cudaMalloc(&p->d_tile, bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
        p->tile_bytes = bytes;
    }
    if (p->tile_host != tp.bytes) {
        p->tile_host = tp.bytes;
        e = cudaMemcpyAsync(p->d_tile, p->tile_host.data(), bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            p->tile_host.clear();
            return set_cuda_error(e);
        }
    }
    p->shape.cluster = L.C;
    p->shape.slots = L.S;
    p->shape.units_per_warp = 0;
    for (int r = 0; r < L.C; ++r) p->shape.units_per_warp = std::max(p->shape.units_per_warp, L.slices[r]);
    p->shape.units_per_warp = (p->shape.units_per_warp + L.warps - 1) / L.warps;
    p->shape.threads = 32 * L.warps;
    p->shape.smem_bytes = L.smem_bytes;
    p->shape.grid = grid;
    p->shape.variant = 3;
    if (M == 0 || p->dry_run) return FTWA_OK;

    TileArgs a;
    fill_args(p, L, tp, static_cast<unsigned char *>(p->d_tile), a);
    a.M = M;
    a.n_steps = n_steps;
    a.rho = reinterpret_cast<float2 *>(rho);
    a.snap = reinterpret_cast<float *>(snap);
    e = cudaLaunchKernelEx(&cfg, kern, a);
    return set_cuda_error(e);
}

}  // namespace ftwa

// Host-only consistency check of the tiled stepper's work decomposition for a
// lattice (no device needed); see include/ftwa.h.
extern "C" int ftwa_debug_tile_check(int32_t n_sites, int32_t n_bonds, const int32_t *bonds, const double *t_bond,
                                     int32_t cluster, int32_t slots, int64_t *violations, char *msg, int32_t msg_len)
{
    using namespace ftwa;
    using namespace ftwa::tile;
    if (n_sites < 2 || n_sites > FTWA_MAX_SITES || n_bonds < 0 || (!bonds && n_bonds) || !violations)
        return FTWA_ERR_INVALID_ARGUMENT;
    if (msg && msg_len > 0) msg[0] = 0;
    Plan p;
    p.N = n_sites;
    p.precision = FTWA_FP32;
    p.bonds.assign(bonds, bonds + 2 * (size_t)n_bonds);
    p.t_bond.assign((size_t)n_bonds, 1.0);
    if (t_bond)
        for (int b = 0; b < n_bonds; ++b) p.t_bond[b] = t_bond[b];
    std::vector<int> deg(n_sites, 0);
    p.bandwidth = 1;
    for (int b = 0; b < n_bonds; ++b) {
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || j >= n_sites || i >= j) return FTWA_ERR_INVALID_ARGUMENT;
        if (++deg[i] > 3 || ++deg[j] > 3) return FTWA_ERR_UNSUPPORTED;
        p.bandwidth = std::max(p.bandwidth, j - i);
    }
    std::vector<Nbr> nb;
    neighbours(&p, nb);
    RowSlots rs;
    row_part_slots(p.N, p.bandwidth, nb, rs);
    // both CTA sizes the stepper launches with
    *violations = 0;
    bool any = false;
    for (int warps : {16, 24}) {
        Layout L;
        if (!build_layout(&p, nb, rs, is_pm1(nb), cluster, slots, warps, L)) continue;
        any = true;
        *violations += check_layout(L, nb, msg, msg_len);
    }
    return any ? FTWA_OK : FTWA_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------------------
// Persistent batched launch over several plans (lattices of different sizes,
// several U): one cluster-launched kernel whose clusters draw (problem, sample
// batch) items from a queue ordered by cost, largest first.
// ---------------------------------------------------------------------------
namespace ftwa {
namespace tile {

struct BatchConfig {
    int C = 0, warps = 0, smem = 0, grid = 0;
    std::vector<Layout> L;
    std::vector<TablePack> tp;
    std::vector<int2> items;
};

static bool batch_config(Plan *const *plans, int n, const int64_t *M, const std::vector<std::vector<Nbr>> &nb,
                         const std::vector<RowSlots> &rs, const std::vector<char> &pm1, int C, int warps,
                         BatchConfig &bc)
{
    bc = BatchConfig();
    bc.C = C;
    bc.warps = warps;
    bc.L.resize(n);
    bc.tp.resize(n);
    std::vector<std::pair<long long, int2>> its;
    for (int i = 0; i < n; ++i) {
        // the smallest group of CTAs (a divisor of C) the problem fits on; the
        // cluster's C / Ci groups then integrate batches of it side by side
        bool ok = false;
        for (int Ci = 1; Ci <= C && !ok; Ci *= 2)
            ok = choose_layout(plans[i], std::max<int64_t>(M[i], 1), nb[i], rs[i], pm1[i] != 0, bc.L[i], Ci, warps,
                               true);
        if (!ok) return false;
        bc.smem = std::max(bc.smem, bc.L[i].smem_bytes);
        pack_tables(bc.L[i], bc.tp[i]);
        const int S = bc.L[i].S, N = plans[i]->N, Ci = bc.L[i].C, groups = C / Ci;
        const long long batches = (M[i] + S - 1) / S;
        const long long items = (batches + groups - 1) / groups;
        for (long long j = 0; j < items; ++j) its.push_back({(long long)S * N * (N + 1) / Ci, int2{i, (int)j}});
    }
    std::stable_sort(its.begin(), its.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    for (auto &x : its) bc.items.push_back(x.second);
    return bc.smem <= 227 * 1024;
}

// Upload a configuration (tables, queue, counter) into one device buffer and
// write the kernel arguments; *mem receives the buffer (owned by the caller).
static int batch_upload(Plan *const *plans, int n, const BatchConfig &bc, void *const *rho, const int64_t *M,
                        int64_t n_steps, void *const *snap, BatchArgs &B, void **mem, cudaStream_t s)
{
    size_t off = 0;
    std::vector<size_t> tab_off(n);
    for (int i = 0; i < n; ++i) {
        tab_off[i] = off;
        off += ((bc.tp[i].bytes.size() + 255) / 256) * 256;
    }
    const size_t items_off = off;
    off += ((bc.items.size() * sizeof(int2) + 255) / 256) * 256;
    const size_t counter_off = off;
    off += 256;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, off);
    if (e != cudaSuccess) return set_cuda_error(e);
    unsigned char *base = static_cast<unsigned char *>(d);
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(base + tab_off[i], bc.tp[i].bytes.data(), bc.tp[i].bytes.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !bc.items.empty())
        e = cudaMemcpyAsync(base + items_off, bc.items.data(), bc.items.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host images are freed with the configuration
    if (e != cudaSuccess) {
        cudaFree(d);
        return set_cuda_error(e);
    }
    std::memset(&B, 0, sizeof(B));
    B.n_items = (int)bc.items.size();
    B.C = bc.C;
    B.items = reinterpret_cast<const int2 *>(base + items_off);
    B.counter = reinterpret_cast<int *>(base + counter_off);
    for (int i = 0; i < n; ++i) {
        fill_args(plans[i], bc.L[i], bc.tp[i], base + tab_off[i], B.prob[i]);
        B.prob[i].M = M[i];
        B.prob[i].n_steps = n_steps;
        B.prob[i].rho = reinterpret_cast<float2 *>(rho[i]);
        B.prob[i].snap = snap ? reinterpret_cast<float *>(snap[i]) : nullptr;
        B.prob[i].force_timeout = 0;
    }
    *mem = d;
    return FTWA_OK;
}

static void (*batch_kernel(int warps))(BatchArgs)
{
    return warps == 16 ? tile_batch_stepper<512> : tile_batch_stepper<768>;
}

// launch configuration of a batch (grid: every co-resident cluster)
static int batch_launch_cfg(const BatchConfig &bc, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr,
                            cudaStream_t s)
{
    auto kern = batch_kernel(bc.warps);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bc.smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    cfg = cudaLaunchConfig_t{};
    cfg.blockDim = dim3(32 * bc.warps, 1, 1);
    cfg.dynamicSmemBytes = bc.smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = bc.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(bc.C, 1, 1);
    int n_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&n_clusters, kern, &cfg);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (n_clusters < 1) return FTWA_ERR_UNSUPPORTED;
    cfg.gridDim = dim3(n_clusters * bc.C, 1, 1);
    return FTWA_OK;
}

}  // namespace tile
}  // namespace ftwa

extern "C" int ftwa_batch_create_persistent(ftwa_plan_t *const *plans, int32_t n, void *const *rho_dev,
                                            const int64_t *M, int64_t n_steps, void *const *snap_dev, int32_t tune,
                                            ftwa_batch_t **out)
{
    using namespace ftwa;
    using namespace ftwa::tile;
    if (!out || !plans || !rho_dev || !M || n < 1 || n > kMaxBatch || n_steps < 0) return FTWA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || M[i] < 0 || (M[i] > 0 && !rho_dev[i])) return FTWA_ERR_INVALID_ARGUMENT;
        if (!tile_supported(plans[i]) || plans[i]->device != plans[0]->device) return FTWA_ERR_UNSUPPORTED;
    }
    std::vector<Plan *> P(plans, plans + n);
    std::vector<std::vector<Nbr>> nb(n);
    std::vector<char> pm1(n);
    std::vector<RowSlots> rs(n);
    for (int i = 0; i < n; ++i) {
        neighbours(P[i], nb[i]);
        pm1[i] = is_pm1(nb[i]) ? 1 : 0;
        plan_row_slots(P[i], nb[i], rs[i]);
    }
    // the smallest cluster size every problem fits
    int C_min = 0;
    for (int C = 1; C <= kMaxCluster && !C_min; C *= 2) {
        BatchConfig bc;
        if (batch_config(P.data(), n, M, nb, rs, pm1, C, 24, bc)) C_min = C;
    }
    if (!C_min) return FTWA_ERR_UNSUPPORTED;
    std::vector<std::pair<int, int>> cands = {{C_min, 24}};
    if (tune) {
        cands.push_back({C_min, 16});
        if (2 * C_min <= kMaxCluster) {
            cands.push_back({2 * C_min, 24});
            cands.push_back({2 * C_min, 16});
        }
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FTWA_ERR_CUDA;
    int rc = FTWA_OK;
    int best = 0;
    if (cands.size() > 1) {
        // autotune: time each candidate on a probe (scratch states of up to 64
        // batches per problem, a few steps)
        std::vector<int64_t> Mp(n);
        std::vector<void *> rp(n, nullptr);
        float best_ms = -1.f;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (size_t c = 0; c < cands.size() && rc == FTWA_OK; ++c) {
            BatchConfig bc;
            if (!batch_config(P.data(), n, M, nb, rs, pm1, cands[c].first, cands[c].second, bc)) continue;
            for (int i = 0; i < n && rc == FTWA_OK; ++i) {
                Mp[i] = std::min<int64_t>(M[i], 64LL * bc.L[i].S);
                cudaFree(rp[i]);
                rp[i] = nullptr;
                if (Mp[i] == 0) continue;
                if (cudaMalloc(&rp[i], (size_t)Mp[i] * 2 * P[i]->N * P[i]->N * 8) != cudaSuccess) rc = FTWA_ERR_OUT_OF_MEMORY;
                else rc = launch_sample(P[i], 12345, 0, Mp[i], rp[i], s);
            }
            if (rc != FTWA_OK) break;
            BatchConfig bp;
            if (!batch_config(P.data(), n, Mp.data(), nb, rs, pm1, cands[c].first, cands[c].second, bp)) continue;
            BatchArgs B;
            void *mem = nullptr;
            rc = batch_upload(P.data(), n, bp, rp.data(), Mp.data(), std::min<int64_t>(n_steps, 10), nullptr, B, &mem, s);
            if (rc != FTWA_OK) break;
            cudaLaunchConfig_t cfg;
            cudaLaunchAttribute attr[1];
            int r2 = batch_launch_cfg(bp, cfg, attr, s);
            if (r2 == FTWA_OK) {
                cudaMemsetAsync(B.counter, 0, sizeof(int), s);
                cudaEventRecord(e0, s);
                cudaError_t e = cudaLaunchKernelEx(&cfg, batch_kernel(bp.warps), B);
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) rc = set_cuda_error(e);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rc == FTWA_OK && (best_ms < 0.f || ms < best_ms)) {
                    best_ms = ms;
                    best = (int)c;
                }
            } else if (r2 != FTWA_ERR_UNSUPPORTED) {
                rc = r2;
            }
            cudaFree(mem);
        }
        for (int i = 0; i < n; ++i) cudaFree(rp[i]);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    BatchConfig bc;
    BatchArgs B;
    void *mem = nullptr;
    if (rc == FTWA_OK && !batch_config(P.data(), n, M, nb, rs, pm1, cands[best].first, cands[best].second, bc))
        rc = FTWA_ERR_UNSUPPORTED;
    if (rc == FTWA_OK) rc = batch_upload(P.data(), n, bc, rho_dev, M, n_steps, snap_dev, B, &mem, s);
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    if (rc == FTWA_OK) rc = batch_launch_cfg(bc, cfg, attr, s);
    ftwa_batch *b = nullptr;
    if (rc == FTWA_OK) {
        b = new (std::nothrow) ftwa_batch();
        if (!b) rc = FTWA_ERR_OUT_OF_MEMORY;
    }
    if (rc == FTWA_OK) {
        // one graph: zero the queue head, then the persistent kernel
        b->n = n;
        b->d_owned = mem;
        mem = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(B.counter, 0, sizeof(int), s);
            cfg.stream = s;
            if (e1 == cudaSuccess) e1 = cudaLaunchKernelEx(&cfg, batch_kernel(bc.warps), B);
            e = cudaStreamEndCapture(s, &b->graph);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) rc = set_cuda_error(e);
        // plan info: the batch's shape
        for (int i = 0; i < n && rc == FTWA_OK; ++i) {
            P[i]->shape.cluster = bc.L[i].C;
            P[i]->shape.slots = bc.L[i].S;
            P[i]->shape.threads = 32 * bc.warps;
            P[i]->shape.smem_bytes = bc.smem;
            P[i]->shape.grid = (int)cfg.gridDim.x;
            P[i]->shape.variant = 3;
        }
    }
    cudaStreamDestroy(s);
    if (mem) cudaFree(mem);
    if (rc != FTWA_OK) {
        if (b) ftwa_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FTWA_OK;
}
