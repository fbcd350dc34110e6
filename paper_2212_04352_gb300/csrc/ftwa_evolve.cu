// Persistent RK4 stepper for the fTWA equation of motion (Eq. 6).
//
// One sample's state (both spins, Hermitian, packed upper triangle) stays
// on chip for the whole integration:
//  - the RK4 stage state lives in shared memory, double-buffered, and for
//    large lattices is split by spin-rows across a thread-block cluster
//    (neighbour rows owned by another CTA are read through distributed
//    shared memory);
//  - the private RK4 registers of every element (y0 and the stage
//    accumulator) and its index metadata live in tensor memory, which the
//    stepper uses as a 256 KB per-SM extension of the register file;
//  - the diagonal Re rho_kk of both spins (the U coupling of Eq. 6) is
//    replicated into every CTA of the cluster at each stage.
// Work unit: 32 consecutive packed elements, one per lane.  A CTA owns a set
// of spin-rows (and, for small lattices, several samples, "slots").
//
// Per element (p, q), p <= q, spin s, the right-hand side of Eq. 6 is
//   k_pq = i [ sum_{k in nb(q)} t_qk rho_pk - sum_{k in nb(p)} t_pk rho_kq
//              + U (Re rho_pp,sbar - Re rho_qq,sbar) rho_pq ]
// with rho_ab = conj(rho_ba) for a > b read from the stored triangle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "ftwa_internal.h"
#include "ptx.cuh"

namespace ftwa {

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

template <typename T>
struct StepArgs {
    const int32_t *nbr;   // [N] k0 | k1 << 8 | k2 << 16 | deg << 24
    const T *tnb;         // [N][4]
    T U, dt, t_uniform;
    int N, C, S, E, buf_bytes, n_units_max, fast_chunk;
    int row_begin[kMaxCluster + 1];
    long long M, n_steps;
    int out_every;
    typename C2<T>::type *rho;   // [M][2][N][N]
    T *snap;                     // [n_out][M][2N] or null
    int *status;
    unsigned long long timeout_ns;
    int force_timeout;
};

struct SmemHeader {
    unsigned long long bar;       // cluster barrier (count = C)
    unsigned long long dead_bar;  // never completes (timeout test hook)
    uint32_t tmem_base;
    int abort;
    int n_units;
    int pad;
};

// Per spin-row descriptor.  base(r) denotes the address of element (p, 0)
// of row r = (s, p) in stage buffer A as if the row were stored in full:
// element (p, q), q >= p, lives at base(r) + q * sizeof(V).
struct __align__(16) RowDesc {
    uint32_t base_local;   // base of this row in the owning CTA (shared::cta)
    uint32_t base_k[3];    // bases of the rows of p's neighbours: shared::cta if
                           // the row is owned by this CTA, else shared::cluster
    int32_t nbp;           // p's neighbour slots (packed as in nbr)
    int32_t p;             // site index
    int32_t remote;        // bit n: neighbour row n lives in another CTA
    int32_t deg;           // number of bonds of p
    uint32_t base_kc[3];   // the same bases as shared::cluster addresses
    uint32_t pad;
};

__device__ __forceinline__ void record_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// Barrier over the cluster (C > 1: mbarrier with a bounded wait; C == 1:
// __syncthreads).  Returns false when the CTA must abort.
template <bool CLUSTER>
__device__ __forceinline__ bool stage_barrier(SmemHeader *h, uint32_t &phase, int C, unsigned long long limit,
                                              int *status)
{
    __syncthreads();
    if constexpr (CLUSTER) {
        const uint32_t bar = smem_addr(&h->bar);
        if ((int)threadIdx.x < C) mbar_arrive_cluster(map_rank(bar, threadIdx.x));
        if (threadIdx.x == 0) {
            if (!mbar_wait_bounded(bar, phase, limit)) {
                h->abort = 1;
                record_status(status, FTWA_ERR_DEVICE_TIMEOUT);
            }
        }
        __syncthreads();
        phase ^= 1u;
    }
    return h->abort == 0;
}

template <typename T, bool CLUSTER>
__device__ __forceinline__ typename C2<T>::type ld_state(uint32_t a)
{
    if constexpr (CLUSTER) return ldc2(a, T());
    else return lds2(a, T());
}

// tensor-memory state words of one element: y0 then acc (WC words each)
template <int WC>
__device__ __forceinline__ void tmem_ld_state(uint32_t ta, uint32_t (&w)[2 * WC])
{
    if constexpr (WC == 2) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "r"(ta) : "memory");
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                     : "r"(ta)
                     : "memory");
    }
}
// wait for the load; the words are in/out operands so no use of them can be
// scheduled before the wait
template <int WC>
__device__ __forceinline__ void tmem_wait_ld_regs(uint32_t (&w)[2 * WC])
{
    if constexpr (WC == 2) {
        asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]) :: "memory");
    } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]), "+r"(w[6]), "+r"(w[7])
                     :: "memory");
    }
}
template <int WC>
__device__ __forceinline__ void tmem_wait_ld_regs2(uint32_t (&w)[2 * WC], uint32_t (&v)[2 * WC])
{
    if constexpr (WC == 2) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3])
                     :: "memory");
    } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]), "+r"(w[6]), "+r"(w[7]),
                       "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
                     :: "memory");
    }
}
template <int WC, typename V>
__device__ __forceinline__ void unpack_state(const uint32_t (&w)[2 * WC], V &y0, V &acc)
{
    if constexpr (WC == 2) {
        y0.x = __uint_as_float(w[0]);
        y0.y = __uint_as_float(w[1]);
        acc.x = __uint_as_float(w[2]);
        acc.y = __uint_as_float(w[3]);
    } else {
        y0.x = __longlong_as_double(((unsigned long long)w[1] << 32) | w[0]);
        y0.y = __longlong_as_double(((unsigned long long)w[3] << 32) | w[2]);
        acc.x = __longlong_as_double(((unsigned long long)w[5] << 32) | w[4]);
        acc.y = __longlong_as_double(((unsigned long long)w[7] << 32) | w[6]);
    }
}

template <int STAGE, typename T, bool CLUSTER, bool UNIFORM_T>
__device__ __forceinline__ void rk4_stage(const StepArgs<T> &a, const RowDesc *s_desc, const uint32_t *s_rowbase,
                                          const uint32_t *s_units, const int32_t *s_nbr, const T *s_t, T *s_diag,
                                          uint32_t diag_s, int n_units, int warp, int lane, uint32_t t_state,
                                          int eps_bytes, int diag_stride, long long b, bool snap_now,
                                          long long snap_row)
{
    using V = typename C2<T>::type;
    constexpr int SZ = sizeof(V);
    constexpr int WC = SZ / 4;
    constexpr int CUR = STAGE & 1;
    const int N = a.N, twoN = 2 * N;
    const uint32_t boff_cur = CUR ? (uint32_t)a.buf_bytes : 0u;
    const uint32_t boff_nxt = CUR ? 0u : (uint32_t)a.buf_bytes;
    const T *dg = s_diag + CUR * diag_stride;
    const T half_dt = a.dt * T(0.5), sixth_dt = a.dt / T(6);
    // y0 and acc of the next unit are loaded from tensor memory while the
    // current unit computes (one tcgen05.ld in flight per warp)
    uint32_t nx[2 * WC];
    tmem_ld_state<WC>(t_state, nx);
    for (int j = 0; j < a.E; ++j) {
        const int u = j * kWarps + warp;
        tmem_wait_ld_regs<WC>(nx);
        V y0, acc;
        unpack_state<WC>(nx, y0, acc);
        __syncwarp();
        if (j + 1 < a.E) tmem_ld_state<WC>(t_state + (uint32_t)((j + 1) * 2 * WC), nx);
        if (u < n_units) {
            const uint32_t unit = s_units[u];
            const int chunk = unit & 7, sr = (unit >> 3) & 511, slot = unit >> 12;
            const RowDesc d = s_desc[sr];
            const int p = d.p, s = sr >= N ? 1 : 0;
            const int q = p + 32 * chunk + lane;
            if (q < N) {
                const uint32_t soff = (uint32_t)(slot * eps_bytes) + boff_cur;
                const uint32_t qoff = soff + (uint32_t)(q * SZ);
                const V own = lds2(d.base_local + qoff, T());
                const int nq = s_nbr[q];
                T hr = T(0), hi = T(0);
                if (chunk >= a.fast_chunk) {
                    // away from the diagonal: every rho_pk (k in nb(q)) and rho_kq
                    // (k in nb(p)) is in the stored triangle; rho_pk is in this
                    // CTA's own row p.  Empty neighbour slots carry zero hopping.
#pragma unroll
                    for (int n = 0; n < 3; ++n) {
                        const int k = (nq >> (8 * n)) & 0xFF;
                        const T t = UNIFORM_T ? (n < (nq >> 24) ? a.t_uniform : T(0)) : s_t[4 * q + n];
                        const V v = lds2(d.base_local + soff + (uint32_t)(k * SZ), T());
                        hr = fma(t, v.x, hr);
                        hi = fma(t, v.y, hi);
                    }
#pragma unroll
                    for (int n = 0; n < 3; ++n) {
                        const T t = UNIFORM_T ? (n < d.deg ? a.t_uniform : T(0)) : s_t[4 * p + n];
                        const V v = CLUSTER ? ldc2(d.base_kc[n] + qoff, T()) : lds2(d.base_k[n] + qoff, T());
                        hr = fma(-t, v.x, hr);
                        hi = fma(-t, v.y, hi);
                    }
                } else {
                    // near the diagonal: entries below it are read as conj(rho_ba)
#pragma unroll
                    for (int n = 0; n < 3; ++n) {
                        const int k = (nq >> (8 * n)) & 0xFF;
                        const T t = UNIFORM_T ? (n < (nq >> 24) ? a.t_uniform : T(0)) : s_t[4 * q + n];
                        V v;
                        if (k >= p) {
                            v = lds2(d.base_local + soff + (uint32_t)(k * SZ), T());
                        } else {
                            v = ld_state<T, CLUSTER>(s_rowbase[s * N + k] + soff + (uint32_t)(p * SZ));
                            v.y = -v.y;
                        }
                        hr = fma(t, v.x, hr);
                        hi = fma(t, v.y, hi);
                    }
#pragma unroll
                    for (int n = 0; n < 3; ++n) {
                        if (n < d.deg) {
                            const int k = (d.nbp >> (8 * n)) & 0xFF;
                            const T t = UNIFORM_T ? a.t_uniform : s_t[4 * p + n];
                            V v;
                            if (k <= q) {
                                if (CLUSTER && ((d.remote >> n) & 1)) v = ldc2(d.base_k[n] + qoff, T());
                                else v = lds2(d.base_k[n] + qoff, T());
                            } else {
                                v = ld_state<T, CLUSTER>(s_rowbase[s * N + q] + soff + (uint32_t)(k * SZ));
                                v.y = -v.y;
                            }
                            hr = fma(-t, v.x, hr);
                            hi = fma(-t, v.y, hi);
                        }
                    }
                }
                // + U (Re rho_pp,sbar - Re rho_qq,sbar) rho_pq
                const T *db = dg + slot * twoN + (1 - s) * N;
                const T g = a.U * (db[p] - db[q]);
                hr = fma(g, own.x, hr);
                hi = fma(g, own.y, hi);
                // k = i (hr + i hi); on the diagonal Eq. 6 is real, so its imaginary
                // part (pure rounding residue) is dropped
                const T kx = -hi, ky = (q == p) ? T(0) : hr;
                V nxt;
                if constexpr (STAGE == 0) {
                    acc.x = kx;
                    acc.y = ky;
                    nxt.x = fma(half_dt, kx, y0.x);
                    nxt.y = fma(half_dt, ky, y0.y);
                } else if constexpr (STAGE < 3) {
                    acc.x = fma(T(2), kx, acc.x);
                    acc.y = fma(T(2), ky, acc.y);
                    const T c = STAGE == 1 ? half_dt : a.dt;
                    nxt.x = fma(c, kx, y0.x);
                    nxt.y = fma(c, ky, y0.y);
                } else {
                    nxt.x = fma(sixth_dt, acc.x + kx, y0.x);
                    nxt.y = fma(sixth_dt, acc.y + ky, y0.y);
                    y0 = nxt;
                }
                sts2(d.base_local + qoff - boff_cur + boff_nxt, nxt);
                if (q == p) {
                    const int di = (CUR ^ 1) * diag_stride + slot * twoN + s * N + p;
                    if constexpr (CLUSTER) {
                        const uint32_t da = diag_s + (uint32_t)(di * (int)sizeof(T));
                        for (int r = 0; r < a.C; ++r) stc1(map_rank(da, r), nxt.x);
                    } else {
                        s_diag[di] = nxt.x;
                    }
                    if (STAGE == 3 && snap_now) {
                        const long long m = b * a.S + slot;
                        if (m < a.M) a.snap[(snap_row * a.M + m) * twoN + s * N + p] = nxt.x;
                    }
                }
            }
        }
        __syncwarp();
        if constexpr (STAGE < 3) tmem_put(t_state + (uint32_t)(j * 2 * WC + WC), acc);
        else tmem_put(t_state + (uint32_t)(j * 2 * WC), y0);
    }
}

template <typename T, bool CLUSTER, bool UNIFORM_T>
__global__ void __launch_bounds__(kThreads, 1) rk4_stepper(const StepArgs<T> a)
{
    using V = typename C2<T>::type;
    constexpr int SZ = sizeof(V);
    constexpr int WC = SZ / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = a.N, S = a.S, C = a.C, twoN = 2 * N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t cid = CLUSTER ? cluster_id_x() : blockIdx.x;
    const uint32_t ncl = CLUSTER ? n_clusters_x() : gridDim.x;

    // ---- shared-memory carve-up (mirrors smem_needed on the host) -----------
    unsigned char *ptr = smem;
    SmemHeader *h = reinterpret_cast<SmemHeader *>(ptr);
    ptr += 64;
    int32_t *s_nbr = reinterpret_cast<int32_t *>(ptr);
    ptr += 4 * 256;
    T *s_t = reinterpret_cast<T *>(ptr);
    ptr += sizeof(T) * 4 * 256;
    RowDesc *s_desc = reinterpret_cast<RowDesc *>(ptr);
    ptr += sizeof(RowDesc) * 2 * 256;
    uint32_t *s_rowbase = reinterpret_cast<uint32_t *>(ptr);
    ptr += 4 * 2 * 256;
    uint32_t *s_units = reinterpret_cast<uint32_t *>(ptr);
    ptr += 4 * ((a.n_units_max + 3) / 4) * 4;
    T *s_diag = reinterpret_cast<T *>(ptr);                        // [2 buf][S][2N]
    ptr += ((sizeof(T) * 2 * S * twoN + 15) / 16) * 16;
    unsigned char *bufA = ptr;
    const uint32_t bufA_s = smem_addr(bufA);
    const uint32_t diag_s = smem_addr(s_diag);
    const int diag_stride = S * twoN;

    const int rb0 = a.row_begin[rank], rb1 = a.row_begin[rank + 1];
    int eps = 0;                      // packed elements per slot of this rank
    for (int sr = rb0; sr < rb1; ++sr) eps += N - (sr % N);
    const int eps_bytes = eps * SZ;

    if (threadIdx.x == 0) {
        h->abort = 0;
        mbar_init(smem_addr(&h->bar), (uint32_t)C);
        mbar_init(smem_addr(&h->dead_bar), 1u);
        fence_mbar_init_cluster();
        // work units: (slot, spin-row, 32-column chunk) of this rank.  Units
        // next to the diagonal (slower path) come first, so that unit u =
        // j * kWarps + warp deals them evenly over the warps.
        int nu = 0;
        for (int pass = 0; pass < 2; ++pass)
            for (int slot = 0; slot < S; ++slot)
                for (int sr = rb0; sr < rb1; ++sr) {
                    const int len = N - sr % N;
                    for (int c = 0; c * 32 < len; ++c)
                        if ((c < a.fast_chunk) == (pass == 0))
                            s_units[nu++] = (uint32_t)c | ((uint32_t)sr << 3) | ((uint32_t)slot << 12);
                }
        h->n_units = nu;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        s_nbr[i] = a.nbr[i];
        for (int n = 0; n < 4; ++n) s_t[4 * i + n] = a.tnb[4 * i + n];
    }
    // row bases (slot 0, buffer A)
    for (int sr = threadIdx.x; sr < twoN; sr += blockDim.x) {
        int owner = 0;
        while (owner + 1 < C && sr >= a.row_begin[owner + 1]) ++owner;
        int off = 0;
        for (int x = a.row_begin[owner]; x < sr; ++x) off += N - (x % N);
        const int p = sr % N;
        // map the row's first stored element (p, p), then shift by -p so that
        // (p, q) is at base + q * SZ (only q >= p is ever addressed)
        const uint32_t start = bufA_s + (uint32_t)(off * SZ);
        s_rowbase[sr] = (CLUSTER ? map_rank(start, owner) : start) - (uint32_t)(p * SZ);
    }
    __syncthreads();
    for (int sr = threadIdx.x; sr < twoN; sr += blockDim.x) {
        const int s = sr / N, p = sr % N;
        RowDesc d;
        d.p = p;
        d.nbp = s_nbr[p];
        d.deg = (d.nbp >> 24) & 0xFF;
        d.remote = 0;
        for (int n = 0; n < 3; ++n) {
            const int k = (d.nbp >> (8 * n)) & 0xFF, r = s * N + k;
            int owner = 0;
            while (owner + 1 < C && r >= a.row_begin[owner + 1]) ++owner;
            d.base_kc[n] = s_rowbase[r];
            if (CLUSTER && owner != (int)rank) {
                d.base_k[n] = s_rowbase[r];
                d.remote |= 1 << n;
            } else {
                int off = 0;
                for (int x = rb0; x < r; ++x) off += N - (x % N);
                d.base_k[n] = bufA_s + (uint32_t)(off * SZ) - (uint32_t)(k * SZ);
            }
        }
        int off = 0;
        for (int x = rb0; x < sr && x < rb1; ++x) off += N - (x % N);
        d.base_local = bufA_s + (uint32_t)(off * SZ) - (uint32_t)(p * SZ);
        d.pad = 0;
        s_desc[sr] = d;
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(&h->tmem_base), kTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if constexpr (CLUSTER) cluster_sync_hw();   // barrier inits visible cluster-wide

    const int n_units = h->n_units;
    const uint32_t t_state = h->tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemColsPerWarp * (warp >> 2));

    uint32_t phase = 0;
    const unsigned long long limit = a.timeout_ns;
    if (a.force_timeout) {
        // test hook: a bounded wait on a barrier that nothing arrives at
        if (threadIdx.x == 0 && !mbar_wait_bounded(smem_addr(&h->dead_bar), 0u, limit)) {
            h->abort = 1;
            record_status(a.status, FTWA_ERR_DEVICE_TIMEOUT);
        }
        __syncthreads();
    }

    const long long n_batches = (a.M + S - 1) / S;
    for (long long b = cid; b < n_batches && h->abort == 0; b += ncl) {
        // ---- load rho(0) ---------------------------------------------------------
        for (int j = 0; j < a.E; ++j) {
            const int u = j * kWarps + warp;
            __syncwarp();
            V v;
            v.x = T(0);
            v.y = T(0);
            if (u < n_units) {
                const uint32_t unit = s_units[u];
                const int chunk = unit & 7, sr = (unit >> 3) & 511, slot = unit >> 12;
                const int p = sr % N, s = sr / N, q = p + 32 * chunk + lane;
                if (q < N) {
                    const long long m = b * S + slot;
                    if (m < a.M) {
                        v = a.rho[((m * 2 + s) * N + p) * (long long)N + q];
                        if (q == p) {
                            v.y = T(0);
                            if (a.snap) a.snap[m * twoN + s * N + p] = v.x;
                        }
                    }
                    sts2(s_desc[sr].base_local + (uint32_t)(slot * eps_bytes + q * SZ), v);
                    if (q == p) {
                        const int di = slot * twoN + s * N + p;
                        if constexpr (CLUSTER) {
                            const uint32_t da = diag_s + (uint32_t)(di * (int)sizeof(T));
                            for (int r = 0; r < C; ++r) stc1(map_rank(da, r), v.x);
                        } else {
                            s_diag[di] = v.x;
                        }
                    }
                }
            }
            __syncwarp();
            tmem_put(t_state + (uint32_t)(j * 2 * WC), v);
        }
        tmem_wait_st();
        if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;

        // ---- RK4 steps -------------------------------------------------------------
        for (long long step = 0; step < a.n_steps && h->abort == 0; ++step) {
            const bool snap_now = a.snap && ((step + 1) % a.out_every == 0);
            const long long snap_row = (step + 1) / a.out_every;
            rk4_stage<0, T, CLUSTER, UNIFORM_T>(a, s_desc, s_rowbase, s_units, s_nbr, s_t, s_diag, diag_s, n_units,
                                                warp, lane, t_state, eps_bytes, diag_stride, b, snap_now, snap_row);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            rk4_stage<1, T, CLUSTER, UNIFORM_T>(a, s_desc, s_rowbase, s_units, s_nbr, s_t, s_diag, diag_s, n_units,
                                                warp, lane, t_state, eps_bytes, diag_stride, b, snap_now, snap_row);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            rk4_stage<2, T, CLUSTER, UNIFORM_T>(a, s_desc, s_rowbase, s_units, s_nbr, s_t, s_diag, diag_s, n_units,
                                                warp, lane, t_state, eps_bytes, diag_stride, b, snap_now, snap_row);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            rk4_stage<3, T, CLUSTER, UNIFORM_T>(a, s_desc, s_rowbase, s_units, s_nbr, s_t, s_diag, diag_s, n_units,
                                                warp, lane, t_state, eps_bytes, diag_stride, b, snap_now, snap_row);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
        }
        if (h->abort) break;

        // ---- write back rho(T) (full Hermitian matrix) ------------------------------
        for (int j = 0; j < a.E; ++j) {
            const int u = j * kWarps + warp;
            __syncwarp();
            V y0;
            tmem_get(t_state + (uint32_t)(j * 2 * WC), y0);
            if (u >= n_units) continue;
            const uint32_t unit = s_units[u];
            const int chunk = unit & 7, sr = (unit >> 3) & 511, slot = unit >> 12;
            const int p = sr % N, s = sr / N, q = p + 32 * chunk + lane;
            const long long m = b * S + slot;
            if (q >= N || m >= a.M) continue;
            if (!(isfinite(y0.x) && isfinite(y0.y))) record_status(a.status, FTWA_ERR_NONFINITE);
            a.rho[((m * 2 + s) * N + p) * (long long)N + q] = y0;
            if (p != q) {
                V c;
                c.x = y0.x;
                c.y = -y0.y;
                a.rho[((m * 2 + s) * N + q) * (long long)N + p] = c;
            }
        }
        __syncwarp();
    }

    // ---- exit: release tensor memory; no CTA leaves while peers may still
    // address its shared memory -------------------------------------------------
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(h->tmem_base, kTmemCols);
    if constexpr (CLUSTER) cluster_sync_hw();
}

// ---------------------------------------------------------------------------
// Banded stepper.  Used when the site ordering has a small bandwidth bw (max
// |i - j| over bonds), as for honeycomb flakes numbered row by row.
//  - Every spin-row p stores columns [max(0, p - bw), N): the upper triangle
//    plus a mirror band of bw entries below the diagonal, kept equal to
//    conj of the transposed entries.  Every read of Eq. 6 is then a direct
//    load; no conjugated reads near the diagonal.
//  - A lane owns one column q = 32 b + lane of a column block b and walks the
//    rows of its work items, so the column's neighbour offsets, hoppings,
//    other-spin diagonal entry and mirror address stay in registers.
//  - Work items (runs of rows of one spin, one column block) are assigned to
//    warps on the host (longest-processing-time first).
// ---------------------------------------------------------------------------
// Stored columns of row p in the banded layout: the upper triangle plus a
// mirror band of bw entries below the diagonal, columns band_lo(p) .. N - 1.
__host__ __device__ __forceinline__ int band_lo(int p, int bw) { return p > bw ? p - bw : 0; }

template <typename T>
struct BandArgs {
    const int32_t *nbr;
    const T *tnb;
    T U, dt, t_uniform;
    int N, bw, C, S, E, k_items, buf_bytes;
    int qoff;                   // first column of block 0 (<= 0): blocks end at the last column
    int row_begin[kMaxCluster + 1];
    const uint32_t *items;      // [C][kWarps][k_items]: count | b << 6 | sr << 9 | slot << 18
    // FIELD: the diagonal field h_pp,s of every stage is tabulated in shared
    // memory (on-site U or a long-range u, plus the time-dependent drive)
    const T *amp;               // [2][N] drive amplitudes, or null
    const T *ftab;              // [n_steps][4][2] (site pulse f, hopping scale m) at the RK4 stage times, or null
    const T *u;                 // [N][N] symmetric interaction of Eq. 1, or null (on-site U)
    long long M, n_steps;
    int out_every;
    typename C2<T>::type *rho;
    T *snap;
    int *status;
    unsigned long long timeout_ns;
    int force_timeout;
};

struct __align__(16) BandRow {
    uint32_t base_local;   // own row p: element (p, k) at base_local + k * SZ (shared::cta)
    uint32_t base_k[3];    // neighbour rows: shared::cluster addresses in a cluster, else shared::cta
    int32_t p, deg, pad0, pad1;
};

__device__ __forceinline__ void cfma(float t, float2 v, float2 &acc) { acc = __ffma2_rn(make_float2(t, t), v, acc); }
__device__ __forceinline__ void cfma(double t, double2 v, double2 &acc)
{
    acc.x = fma(t, v.x, acc.x);
    acc.y = fma(t, v.y, acc.y);
}

template <int STAGE, typename T, bool CLUSTER, bool UNIFORM_T, bool FIELD>
__device__ __forceinline__ void band_stage(unsigned char *smem, const BandArgs<T> &a, const BandRow *s_row,
                                           const uint32_t *s_rowbase,
                                           const uint32_t *my_items, const int32_t *s_nbr, const T *s_t, T *s_diag,
                                           uint32_t diag_s, int lane, uint32_t t_state, int eps_bytes,
                                           int diag_stride, long long b, bool snap_now, long long snap_row,
                                           const T *s_field, T ms)
{
    using V = typename C2<T>::type;
    constexpr int SZ = sizeof(V);
    constexpr int WC = SZ / 4;
    constexpr int CUR = STAGE & 1;
    const int N = a.N, twoN = 2 * N;
    const uint32_t boff_cur = CUR ? (uint32_t)a.buf_bytes : 0u;
    const uint32_t boff_nxt = CUR ? 0u : (uint32_t)a.buf_bytes;
    const T *dg = s_diag + CUR * diag_stride;
    const T half_dt = a.dt * T(0.5), sixth_dt = a.dt / T(6);
    // local shared-memory accesses go through the __shared__ array (plain
    // loads the compiler can schedule); cluster accesses use PTX
    const uint32_t sbase = smem_addr(smem);
    auto ld_local = [&](uint32_t addr) -> V { return *reinterpret_cast<const V *>(smem + (addr - sbase)); };
    auto st_local = [&](uint32_t addr, V v) { *reinterpret_cast<V *>(smem + (addr - sbase)) = v; };
    int e = 0;
    for (int it = 0; it < a.k_items; ++it) {
        const uint32_t item = my_items[it];
        if (item == 0xFFFFFFFFu) break;
        const int count = item & 63, blk = (item >> 6) & 7, sr0 = (item >> 9) & 511, slot = item >> 18;
        const int s = sr0 >= N ? 1 : 0;
        const int q = a.qoff + 32 * blk + lane;
        const bool qa = q < N;
        const int qc = q < 0 ? 0 : (qa ? q : N - 1);
        // per-column registers for the whole item
        const int nq = s_nbr[qc];
        uint32_t koff[3];
        T tq[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            koff[n] = (uint32_t)(((nq >> (8 * n)) & 0xFF) * SZ);
            tq[n] = UNIFORM_T ? (n < (nq >> 24) ? a.t_uniform : T(0)) : s_t[4 * qc + n];
        }
        const uint32_t soff = (uint32_t)(slot * eps_bytes);
        const uint32_t qsz = (uint32_t)(qc * SZ);
        const uint32_t mirror = s_rowbase[s * N + qc] + soff + boff_nxt;
        const T *dgo = dg + slot * twoN + (1 - s) * N;       // other spin's diagonal
        const T dq = dgo[qc];
        const T *fld = FIELD ? s_field + slot * twoN + s * N : nullptr;   // this spin's diagonal field
        const T fq = FIELD ? fld[qc] : T(0);
        // rows are processed two at a time: independent work for the same warp
        for (int r = 0; r < count; r += 2, e += 2) {
            const bool two = r + 1 < count;
            const int e1 = two ? e + 1 : e;
            uint32_t w0[2 * WC], w1[2 * WC];
            __syncwarp();
            tmem_ld_state<WC>(t_state + (uint32_t)(e * 2 * WC), w0);
            tmem_ld_state<WC>(t_state + (uint32_t)(e1 * 2 * WC), w1);
            tmem_wait_ld_regs2<WC>(w0, w1);
            V y0[2], acc[2];
            unpack_state<WC>(w0, y0[0], acc[0]);
            unpack_state<WC>(w1, y0[1], acc[1]);
            const BandRow d0 = s_row[sr0 + r];
            const BandRow d1 = s_row[sr0 + (two ? r + 1 : r)];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const BandRow &d = i == 0 ? d0 : d1;
                const int p = d.p;
                // every lane computes (inactive lanes on clamped, valid
                // addresses); only the stores are predicated
                const bool active = qa && q >= p && (i == 0 || two);
                const uint32_t rb = d.base_local + soff + boff_cur;
                const V own = lds2(rb + qsz, T());
                V h;
                h.x = T(0);
                h.y = T(0);
                // + sum_{k in nb(q)} t_qk rho_pk   (row p, this CTA)
#pragma unroll
                for (int n = 0; n < 3; ++n) cfma(tq[n], lds2(rb + koff[n], T()), h);
                // - sum_{k in nb(p)} t_pk rho_kq
#pragma unroll
                for (int n = 0; n < 3; ++n) {
                    const T t = UNIFORM_T ? (n < d.deg ? a.t_uniform : T(0)) : s_t[4 * p + n];
                    const uint32_t ad = d.base_k[n] + soff + boff_cur + qsz;
                    cfma(-t, CLUSTER ? ldc2(ad, T()) : lds2(ad, T()), h);
                }
                // (FIELD: every hopping scaled by m(t_stage))
                if constexpr (FIELD) {
                    h.x *= ms;
                    h.y *= ms;
                }
                // + U (Re rho_pp,sbar - Re rho_qq,sbar) rho_pq
                // (FIELD: + (h_pp,s - h_qq,s) rho_pq from the tabulated field)
                T coef;
                if constexpr (FIELD) coef = fld[p] - fq;
                else coef = a.U * (dgo[p] - dq);
                cfma(coef, own, h);
                // k = i h; the diagonal of Eq. 6 is real (its imaginary part is
                // rounding residue and is dropped)
                V kk;
                kk.x = -h.y;
                kk.y = (q == p) ? T(0) : h.x;
                V nxt;
                if constexpr (STAGE == 0) {
                    acc[i] = kk;
                    nxt.x = fma(half_dt, kk.x, y0[i].x);
                    nxt.y = fma(half_dt, kk.y, y0[i].y);
                } else if constexpr (STAGE < 3) {
                    acc[i].x = fma(T(2), kk.x, acc[i].x);
                    acc[i].y = fma(T(2), kk.y, acc[i].y);
                    const T c = STAGE == 1 ? half_dt : a.dt;
                    nxt.x = fma(c, kk.x, y0[i].x);
                    nxt.y = fma(c, kk.y, y0[i].y);
                } else {
                    nxt.x = fma(sixth_dt, acc[i].x + kk.x, y0[i].x);
                    nxt.y = fma(sixth_dt, acc[i].y + kk.y, y0[i].y);
                    y0[i] = nxt;
                }
                if (active) sts2(d.base_local + soff + boff_nxt + qsz, nxt);
                if (active && q != p && q - p <= a.bw) {
                    // mirror entry (q, p) = conj(rho_pq) in row q
                    V c;
                    c.x = nxt.x;
                    c.y = -nxt.y;
                    if constexpr (CLUSTER) stc2(mirror + (uint32_t)(p * SZ), c);
                    else sts2(mirror + (uint32_t)(p * SZ), c);
                }
                if (active && q == p) {
                    const int di = (CUR ^ 1) * diag_stride + slot * twoN + s * N + p;
                    if constexpr (CLUSTER) {
                        const uint32_t da = diag_s + (uint32_t)(di * (int)sizeof(T));
                        for (int rr = 0; rr < a.C; ++rr) stc1(map_rank(da, rr), nxt.x);
                    } else {
                        s_diag[di] = nxt.x;
                    }
                    if (STAGE == 3 && snap_now) {
                        const long long m = b * a.S + slot;
                        if (m < a.M) a.snap[(snap_row * a.M + m) * twoN + s * N + p] = nxt.x;
                    }
                }
            }
            __syncwarp();
            if constexpr (STAGE < 3) {
                tmem_put(t_state + (uint32_t)(e * 2 * WC + WC), acc[0]);
                if (two) tmem_put(t_state + (uint32_t)(e1 * 2 * WC + WC), acc[1]);
            } else {
                tmem_put(t_state + (uint32_t)(e * 2 * WC), y0[0]);
                if (two) tmem_put(t_state + (uint32_t)(e1 * 2 * WC), y0[1]);
            }
        }
        e -= (count & 1);   // an odd item consumed one slot, not two
    }
}

// FIELD: the diagonal field of the coming stage for every slot and spin,
//   h_pp,s = sum_k u_pk (Re rho_kk,sbar + 1/2)     (long-range u of Eq. 1)
//          = U (Re rho_pp,sbar + 1/2)               (on-site U)
//          + amp_s,p f(t_stage)                     (time-dependent drive),
// from the stage's diagonal buffer dg [S][2N]; each CTA of a cluster holds
// all diagonals.  On-site U: every CTA computes the whole table.  Long-range
// u: in a cluster the rows are split over the CTAs, each storing its rows
// into every CTA's table (the caller then meets the cluster barrier), so that
// u is read from L2 once per cluster and stage.  Ends with a CTA barrier.
template <typename T, bool CLUSTER>
__device__ __forceinline__ void diag_field(const BandArgs<T> &a, const T *dg, const T *s_amp, T f, T *s_field,
                                           uint32_t field_s, uint32_t rank)
{
    const int N = a.N, twoN = 2 * N;
    if (a.u) {
        // warp w takes rows r = w, w + n_warps, ... (r = slot * N + p) four at
        // a time: lanes over k (coalesced rows of u), eight independent
        // accumulators, one shuffle reduction per group of four rows
        constexpr int RG = 4;
        const int lane = threadIdx.x & 31;
        const int warp = (CLUSTER ? (int)rank * (int)(blockDim.x >> 5) : 0) + (int)(threadIdx.x >> 5);
        const int n_warps = (CLUSTER ? a.C : 1) * (int)(blockDim.x >> 5);
        const int rows = a.S * N;
        for (int r0 = warp; r0 < rows; r0 += RG * n_warps) {
            T up[RG], dn[RG];
            int rr[RG];
#pragma unroll
            for (int g = 0; g < RG; ++g) {
                rr[g] = r0 + g * n_warps;
                up[g] = T(0);
                dn[g] = T(0);
            }
            for (int k = lane; k < N; k += 32) {
#pragma unroll
                for (int g = 0; g < RG; ++g) {
                    const int r = rr[g] < rows ? rr[g] : rows - 1;
                    const int slot = r / N, p = r % N;
                    const T *d = dg + slot * twoN;
                    const T u = a.u[(size_t)p * N + k];
                    up[g] = fma(u, d[N + k] + T(0.5), up[g]);   // spin up feels the dn density
                    dn[g] = fma(u, d[k] + T(0.5), dn[g]);
                }
            }
#pragma unroll
            for (int g = 0; g < RG; ++g)
                for (int o = 16; o > 0; o >>= 1) {
                    up[g] += __shfl_xor_sync(0xffffffffu, up[g], o);
                    dn[g] += __shfl_xor_sync(0xffffffffu, dn[g], o);
                }
            if (lane == 0) {
#pragma unroll
                for (int g = 0; g < RG; ++g) {
                    if (rr[g] >= rows) continue;
                    const int slot = rr[g] / N, p = rr[g] % N;
                    const T vu = fma(s_amp[p], f, up[g]), vd = fma(s_amp[N + p], f, dn[g]);
                    if constexpr (CLUSTER) {
                        const uint32_t au = field_s + (uint32_t)((slot * twoN + p) * (int)sizeof(T));
                        const uint32_t ad = field_s + (uint32_t)((slot * twoN + N + p) * (int)sizeof(T));
                        for (int c = 0; c < a.C; ++c) {
                            stc1(map_rank(au, (uint32_t)c), vu);
                            stc1(map_rank(ad, (uint32_t)c), vd);
                        }
                    } else {
                        s_field[slot * twoN + p] = vu;
                        s_field[slot * twoN + N + p] = vd;
                    }
                }
            }
        }
    } else {
        for (int i = threadIdx.x; i < a.S * twoN; i += blockDim.x) {
            const int slot = i / twoN, sp = i % twoN, s = sp / N, p = sp % N;
            s_field[i] = fma(s_amp[sp], f, a.U * (dg[slot * twoN + (1 - s) * N + p] + T(0.5)));
        }
    }
    __syncthreads();
}

template <typename T, bool CLUSTER, bool UNIFORM_T, bool FIELD>
__global__ void __launch_bounds__(kThreads, 1) band_stepper(const BandArgs<T> a)
{
    using V = typename C2<T>::type;
    constexpr int SZ = sizeof(V);
    constexpr int WC = SZ / 4;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = a.N, S = a.S, C = a.C, twoN = 2 * N, bw = a.bw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t cid = CLUSTER ? cluster_id_x() : blockIdx.x;
    const uint32_t ncl = CLUSTER ? n_clusters_x() : gridDim.x;

    // shared-memory carve-up (mirrors band_smem on the host)
    unsigned char *ptr = smem;
    SmemHeader *h = reinterpret_cast<SmemHeader *>(ptr);
    ptr += 64;
    BandRow *s_row = reinterpret_cast<BandRow *>(ptr);
    ptr += sizeof(BandRow) * twoN;
    int32_t *s_nbr = reinterpret_cast<int32_t *>(ptr);
    ptr += 16 * ((4 * N + 15) / 16);
    T *s_t = reinterpret_cast<T *>(ptr);
    ptr += 16 * ((sizeof(T) * 4 * N + 15) / 16);
    uint32_t *s_rowbase = reinterpret_cast<uint32_t *>(ptr);
    ptr += 16 * ((4 * twoN + 15) / 16);
    T *s_diag = reinterpret_cast<T *>(ptr);
    ptr += 16 * ((sizeof(T) * 2 * S * twoN + 15) / 16);
    T *s_amp = nullptr, *s_field = nullptr;
    if constexpr (FIELD) {
        s_amp = reinterpret_cast<T *>(ptr);                   // [2N]
        ptr += 16 * ((sizeof(T) * twoN + 15) / 16);
        s_field = reinterpret_cast<T *>(ptr);                 // [S][2N]
        ptr += 16 * ((sizeof(T) * S * twoN + 15) / 16);
    }
    const uint32_t bufA_s = smem_addr(ptr);
    const uint32_t diag_s = smem_addr(s_diag);
    const uint32_t field_s = FIELD ? smem_addr(s_field) : 0u;
    const int diag_stride = S * twoN;

    const int rb0 = a.row_begin[rank], rb1 = a.row_begin[rank + 1];
    int eps = 0;                       // stored elements per slot of this rank
    for (int sr = rb0; sr < rb1; ++sr) eps += N - band_lo(sr % N, bw);
    const int eps_bytes = eps * SZ;

    if (threadIdx.x == 0) {
        h->abort = 0;
        mbar_init(smem_addr(&h->bar), (uint32_t)C);
        mbar_init(smem_addr(&h->dead_bar), 1u);
        fence_mbar_init_cluster();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        s_nbr[i] = a.nbr[i];
        for (int n = 0; n < 4; ++n) s_t[4 * i + n] = a.tnb[4 * i + n];
    }
    if constexpr (FIELD)
        for (int i = threadIdx.x; i < twoN; i += blockDim.x) s_amp[i] = a.amp ? a.amp[i] : T(0);
    // row bases: element (p, k) of spin-row sr (slot 0, buffer A) at base + k * SZ
    for (int sr = threadIdx.x; sr < twoN; sr += blockDim.x) {
        int owner = 0;
        while (owner + 1 < C && sr >= a.row_begin[owner + 1]) ++owner;
        int off = 0;
        for (int x = a.row_begin[owner]; x < sr; ++x) off += N - band_lo(x % N, bw);
        const int p = sr % N, lo = band_lo(p, bw);
        const uint32_t start = bufA_s + (uint32_t)(off * SZ);   // element (p, lo)
        s_rowbase[sr] = (CLUSTER ? map_rank(start, owner) : start) - (uint32_t)(lo * SZ);
    }
    __syncthreads();
    for (int sr = threadIdx.x; sr < twoN; sr += blockDim.x) {
        const int s = sr / N, p = sr % N;
        BandRow d;
        d.p = p;
        const int nbp = s_nbr[p];
        d.deg = (nbp >> 24) & 0xFF;
        for (int n = 0; n < 3; ++n) d.base_k[n] = s_rowbase[s * N + ((nbp >> (8 * n)) & 0xFF)];
        int off = 0;
        for (int x = rb0; x < sr && x < rb1; ++x) off += N - band_lo(x % N, bw);
        const int lo = band_lo(p, bw);
        d.base_local = bufA_s + (uint32_t)(off * SZ) - (uint32_t)(lo * SZ);
        d.pad0 = 0;
        d.pad1 = 0;
        s_row[sr] = d;
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(&h->tmem_base), kTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if constexpr (CLUSTER) cluster_sync_hw();

    const uint32_t t_state = h->tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemColsPerWarp * (warp >> 2));
    const uint32_t *my_items = a.items + ((size_t)rank * kWarps + warp) * a.k_items;

    uint32_t phase = 0;
    const unsigned long long limit = a.timeout_ns;
    if (a.force_timeout) {
        if (threadIdx.x == 0 && !mbar_wait_bounded(smem_addr(&h->dead_bar), 0u, limit)) {
            h->abort = 1;
            record_status(a.status, FTWA_ERR_DEVICE_TIMEOUT);
        }
        __syncthreads();
    }

    const long long n_batches = (a.M + S - 1) / S;
    for (long long b = cid; b < n_batches && h->abort == 0; b += ncl) {
        // ---- load: stored elements of own rows (upper part and mirror band) ----
        for (int slot = 0; slot < S; ++slot) {
            const long long m = b * S + slot;
            for (int sr = rb0 + warp; sr < rb1; sr += kWarps) {
                const int s = sr / N, p = sr % N, lo = band_lo(p, bw);
                const uint32_t base = s_row[sr].base_local + (uint32_t)(slot * eps_bytes);
                for (int k = lo + lane; k < N; k += 32) {
                    V v;
                    v.x = T(0);
                    v.y = T(0);
                    if (m < a.M) {
                        if (k >= p) {
                            v = a.rho[((m * 2 + s) * N + p) * (long long)N + k];
                        } else {
                            v = a.rho[((m * 2 + s) * N + k) * (long long)N + p];
                            v.y = -v.y;
                        }
                    }
                    if (k == p) {
                        v.y = T(0);
                        if (a.snap && m < a.M) a.snap[m * twoN + s * N + p] = v.x;
                        const int di = slot * twoN + s * N + p;
                        if constexpr (CLUSTER) {
                            const uint32_t da = diag_s + (uint32_t)(di * (int)sizeof(T));
                            for (int rr = 0; rr < C; ++rr) stc1(map_rank(da, rr), v.x);
                        } else {
                            s_diag[di] = v.x;
                        }
                    }
                    sts2(base + (uint32_t)(k * SZ), v);
                }
            }
        }
        // y0 of computed elements into tensor memory
        {
            int e = 0;
            for (int it = 0; it < a.k_items; ++it) {
                const uint32_t item = my_items[it];
                if (item == 0xFFFFFFFFu) break;
                const int count = item & 63, blk = (item >> 6) & 7, sr0 = (item >> 9) & 511, slot = item >> 18;
                const int s = sr0 >= N ? 1 : 0;
                const int q = a.qoff + 32 * blk + lane;
                const long long m = b * S + slot;
                for (int r = 0; r < count; ++r, ++e) {
                    const int p = (sr0 + r) % N;
                    V v;
                    v.x = T(0);
                    v.y = T(0);
                    if (q < N && q >= p && m < a.M) {
                        v = a.rho[((m * 2 + s) * N + p) * (long long)N + q];
                        if (q == p) v.y = T(0);
                    }
                    __syncwarp();
                    tmem_put(t_state + (uint32_t)(e * 2 * WC), v);
                }
            }
        }
        tmem_wait_st();
        if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;

        for (long long step = 0; step < a.n_steps && h->abort == 0; ++step) {
            const bool snap_now = a.snap && ((step + 1) % a.out_every == 0);
            const long long snap_row = (step + 1) / a.out_every;
            T fd[4] = {T(0), T(0), T(0), T(0)}, md[4] = {T(1), T(1), T(1), T(1)};
            if constexpr (FIELD)
                if (a.ftab)
                    for (int k = 0; k < 4; ++k) {
                        fd[k] = a.ftab[2 * (4 * step + k)];
                        md[k] = a.ftab[2 * (4 * step + k) + 1];
                    }
            if constexpr (FIELD) {
                diag_field<T, CLUSTER>(a, s_diag + (0 & 1) * diag_stride, s_amp, fd[0], s_field, field_s, rank);
                if (CLUSTER && a.u && !stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            }
            band_stage<0, T, CLUSTER, UNIFORM_T, FIELD>(smem, a, s_row, s_rowbase, my_items, s_nbr, s_t, s_diag,
                                                        diag_s, lane, t_state, eps_bytes, diag_stride, b, snap_now,
                                                        snap_row, s_field, md[0]);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            if constexpr (FIELD) {
                diag_field<T, CLUSTER>(a, s_diag + (1 & 1) * diag_stride, s_amp, fd[1], s_field, field_s, rank);
                if (CLUSTER && a.u && !stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            }
            band_stage<1, T, CLUSTER, UNIFORM_T, FIELD>(smem, a, s_row, s_rowbase, my_items, s_nbr, s_t, s_diag,
                                                        diag_s, lane, t_state, eps_bytes, diag_stride, b, snap_now,
                                                        snap_row, s_field, md[1]);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            if constexpr (FIELD) {
                diag_field<T, CLUSTER>(a, s_diag + (2 & 1) * diag_stride, s_amp, fd[2], s_field, field_s, rank);
                if (CLUSTER && a.u && !stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            }
            band_stage<2, T, CLUSTER, UNIFORM_T, FIELD>(smem, a, s_row, s_rowbase, my_items, s_nbr, s_t, s_diag,
                                                        diag_s, lane, t_state, eps_bytes, diag_stride, b, snap_now,
                                                        snap_row, s_field, md[2]);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            if constexpr (FIELD) {
                diag_field<T, CLUSTER>(a, s_diag + (3 & 1) * diag_stride, s_amp, fd[3], s_field, field_s, rank);
                if (CLUSTER && a.u && !stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            }
            band_stage<3, T, CLUSTER, UNIFORM_T, FIELD>(smem, a, s_row, s_rowbase, my_items, s_nbr, s_t, s_diag,
                                                        diag_s, lane, t_state, eps_bytes, diag_stride, b, snap_now,
                                                        snap_row, s_field, md[3]);
            tmem_wait_st();
            if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
        }
        if (h->abort) break;

        // ---- write back rho(T) (full Hermitian matrix) ------------------------------
        {
            int e = 0;
            for (int it = 0; it < a.k_items; ++it) {
                const uint32_t item = my_items[it];
                if (item == 0xFFFFFFFFu) break;
                const int count = item & 63, blk = (item >> 6) & 7, sr0 = (item >> 9) & 511, slot = item >> 18;
                const int s = sr0 >= N ? 1 : 0;
                const int q = a.qoff + 32 * blk + lane;
                const long long m = b * S + slot;
                for (int r = 0; r < count; ++r, ++e) {
                    const int p = (sr0 + r) % N;
                    __syncwarp();
                    V y0;
                    tmem_get(t_state + (uint32_t)(e * 2 * WC), y0);
                    if (q < N && q >= p && m < a.M) {
                        if (!(isfinite(y0.x) && isfinite(y0.y))) record_status(a.status, FTWA_ERR_NONFINITE);
                        a.rho[((m * 2 + s) * N + p) * (long long)N + q] = y0;
                        if (p != q) {
                            V cj;
                            cj.x = y0.x;
                            cj.y = -y0.y;
                            a.rho[((m * 2 + s) * N + q) * (long long)N + p] = cj;
                        }
                    }
                }
            }
        }
        __syncwarp();
        // the next batch overwrites both stage buffers' own rows; peers read
        // this CTA's rows only after the post-load barrier
        if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
    }

    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc(h->tmem_base, kTmemCols);
    if constexpr (CLUSTER) cluster_sync_hw();
}

// ---------------------------------------------------------------------------
// Host side: launch-shape selection and launch.
// ---------------------------------------------------------------------------
static int smem_needed(int N, int S, int real_bytes, int n_units, int buf_bytes)
{
    int b = 64 + 4 * 256 + real_bytes * 4 * 256 + (int)sizeof(RowDesc) * 2 * 256 + 4 * 2 * 256;
    b += 4 * ((n_units + 3) / 4) * 4;
    b += ((real_bytes * 2 * S * 2 * N + 15) / 16) * 16;
    b += 2 * buf_bytes;
    return b;
}

// Split the 2N spin-rows into C contiguous ranges of balanced cost.  Row p of
// spin s has N - p packed elements in ceil((N - p)/32) work units; units next
// to the diagonal take the slower conj-reading path, weighted 1.5.
static double row_cost(int N, int sr, int fast_chunk)
{
    const int len = N - sr % N, units = (len + 31) / 32;
    return units + 0.5 * std::min(units, fast_chunk);
}

static void split_rows(int N, int C, int fast_chunk, int *rb)
{
    double total = 0;
    for (int sr = 0; sr < 2 * N; ++sr) total += row_cost(N, sr, fast_chunk);
    rb[0] = 0;
    int sr = 0;
    double acc = 0;
    for (int r = 1; r < C; ++r) {
        const double target = total * r / C;
        while (sr < 2 * N && acc + 0.5 * row_cost(N, sr, fast_chunk) < target) {
            acc += row_cost(N, sr, fast_chunk);
            ++sr;
        }
        rb[r] = sr;
    }
    rb[C] = 2 * N;
}

int choose_stepper_shape(Plan *p, int64_t M, StepperShape *out)
{
    const int N = p->N;
    const int real_bytes = p->precision == FTWA_FP64 ? 8 : 4;
    const int elem_bytes = 2 * real_bytes;
    const int WC = elem_bytes / 4;
    const int max_smem = 227 * 1024;
    const int sm = p->sm_count > 0 ? p->sm_count : 1;
    for (int C = 1; C <= kMaxCluster; C *= 2) {
        if (p->cluster_override && C != p->cluster_override) continue;
        StepperShape sh;
        sh.cluster = C;
        split_rows(N, C, (p->bandwidth + 31) / 32, sh.row_begin);
        int eps_max = 0, upr_max = 0;   // elements and 32-column units per slot, max over ranks
        for (int r = 0; r < C; ++r) {
            int eps = 0, upr = 0;
            for (int sr = sh.row_begin[r]; sr < sh.row_begin[r + 1]; ++sr) {
                eps += N - sr % N;
                upr += (N - sr % N + 31) / 32;
            }
            eps_max = std::max(eps_max, eps);
            upr_max = std::max(upr_max, upr);
        }
        if (eps_max == 0) continue;
        // slots: as many samples per CTA as useful (C == 1 only), bounded by
        // tensor-memory and shared-memory capacity
        int want = 1;
        if (C == 1) {
            long long w = (M + sm - 1) / sm;
            want = (int)std::max<long long>(1, std::min<long long>(w, 4096));
        }
        int best = 0;
        for (int S = 1; S <= want; ++S) {
            const int units = S * upr_max;
            const int E = (units + kWarps - 1) / kWarps;
            if (2 * E * WC > kTmemColsPerWarp) break;
            const int buf = ((S * eps_max * elem_bytes + 15) / 16) * 16;
            if (smem_needed(N, S, real_bytes, units, buf) > max_smem) break;
            best = S;
        }
        if (best == 0) continue;
        sh.slots = best;
        sh.n_units = best * upr_max;
        sh.units_per_warp = (sh.n_units + kWarps - 1) / kWarps;
        sh.buf_bytes = ((best * eps_max * elem_bytes + 15) / 16) * 16;
        sh.smem_bytes = std::max(kMinSmem, smem_needed(N, best, real_bytes, sh.n_units, sh.buf_bytes));
        const long long batches = (M + best - 1) / best;
        const int max_groups = std::max(1, sm / C);
        sh.grid = (int)std::min<long long>(std::max<long long>(batches, 1), max_groups) * C;
        *out = sh;
        return FTWA_OK;
    }
    return FTWA_ERR_UNSUPPORTED;
}

template <typename T, bool CLUSTER, bool UNIFORM_T>
static int launch_t(Plan *p, const StepperShape &sh, void *rho, int64_t M, int64_t n_steps, void *snap,
                    cudaStream_t s)
{
    StepArgs<T> a{};
    a.nbr = p->d_nbr;
    a.tnb = std::is_same<T, double>::value ? reinterpret_cast<const T *>(p->d_t64)
                                           : reinterpret_cast<const T *>(p->d_t32);
    a.U = (T)p->U;
    a.dt = (T)p->dt;
    a.t_uniform = p->t_bond.empty() ? T(0) : (T)p->t_bond[0];
    a.N = p->N;
    a.C = sh.cluster;
    a.S = sh.slots;
    a.E = sh.units_per_warp;
    a.buf_bytes = sh.buf_bytes;
    a.n_units_max = sh.n_units;
    a.fast_chunk = (p->bandwidth + 31) / 32;
    for (int i = 0; i <= kMaxCluster; ++i) a.row_begin[i] = sh.row_begin[i];
    a.M = M;
    a.n_steps = n_steps;
    a.out_every = p->out_every;
    a.rho = reinterpret_cast<typename C2<T>::type *>(rho);
    a.snap = reinterpret_cast<T *>(snap);
    a.status = p->d_status;
    a.timeout_ns = p->timeout_ns;
    a.force_timeout = p->force_timeout;
    auto kern = rk4_stepper<T, CLUSTER, UNIFORM_T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem_bytes);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(sh.grid, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = sh.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (CLUSTER) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = sh.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        na = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return set_cuda_error(e);
    return FTWA_OK;
}

template <typename T, bool CLUSTER>
static int dispatch_t(Plan *p, StepperShape &sh, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s)
{
    if (CLUSTER) {
        // clamp the grid to the clusters that can be co-resident
        auto kern = p->uniform_t ? rk4_stepper<T, true, true> : rk4_stepper<T, true, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem_bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(sh.grid, 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = sh.smem_bytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = sh.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n_clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&n_clusters, kern, &cfg);
        if (e != cudaSuccess) return set_cuda_error(e);
        if (n_clusters < 1) return FTWA_ERR_UNSUPPORTED;
        sh.grid = std::min(sh.grid, n_clusters * sh.cluster);
    }
    p->shape = sh;
    p->shape.variant = 2;
    if (M == 0 || p->dry_run) return FTWA_OK;
    return p->uniform_t ? launch_t<T, CLUSTER, true>(p, sh, rho, M, n_steps, snap, s)
                        : launch_t<T, CLUSTER, false>(p, sh, rho, M, n_steps, snap, s);
}

// ---- banded stepper: shape and work items ------------------------------------
// Stored elements of spin-row sr: columns band_lo(p) .. N - 1.
static int band_row_len(int N, int bw, int sr)
{
    return N - band_lo(sr % N, bw);
}

// Column blocks of 32 columns end at the last column, so that only the first
// block is ragged and only the first rows reach it (blocks aligned at column 0
// would leave the last block ragged for every row).
static int band_nblk(int N) { return (N + 31) / 32; }
static int band_qoff(int N) { return N - 32 * band_nblk(N); }
// first column block holding an element q >= p of row p
static int band_first_blk(int p, int qoff) { return (p - qoff) / 32; }

// Work items of one rank: runs of <= R consecutive spin-rows of one spin with
// at least one element in column block b, for every block and slot; assigned
// to warps longest-first under the tensor-memory cap.
static bool band_items(int N, int S, int rb0, int rb1, int e_cap, int R, std::vector<uint32_t> &out, int &E, int &K)
{
    const int nblk = band_nblk(N), qoff = band_qoff(N);
    std::vector<std::pair<int, uint32_t>> items;   // (rows, packed)
    for (int slot = 0; slot < S; ++slot)
        for (int b = 0; b < nblk; ++b)
            for (int s = 0; s < 2; ++s) {
                const int lo = std::max(rb0, s * N), hi = std::min(rb1, s * N + N);
                // rows with p <= qoff + 32 (b + 1) - 1
                const int last = std::min(hi, s * N + std::min(N, qoff + 32 * (b + 1)));
                for (int sr = lo; sr < last;) {
                    const int cnt = std::min(R, last - sr);
                    items.push_back({cnt, (uint32_t)cnt | ((uint32_t)b << 6) | ((uint32_t)sr << 9) | ((uint32_t)slot << 18)});
                    sr += cnt;
                }
            }
    std::stable_sort(items.begin(), items.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<int> load(kWarps, 0);
    std::vector<std::vector<uint32_t>> per(kWarps);
    for (const auto &it : items) {
        int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        if (load[w] + it.first > e_cap) return false;
        load[w] += it.first;
        per[w].push_back(it.second);
    }
    E = *std::max_element(load.begin(), load.end());
    K = 1;
    for (auto &v : per) K = std::max<int>(K, (int)v.size());
    out.assign((size_t)kWarps * K, 0xFFFFFFFFu);
    for (int w = 0; w < kWarps; ++w)
        for (size_t i = 0; i < per[w].size(); ++i) out[(size_t)w * K + i] = per[w][i];
    return true;
}

static int band_smem(int N, int S, int real_bytes, int buf_bytes, bool field)
{
    auto r16 = [](int x) { return 16 * ((x + 15) / 16); };
    int b = 64 + (int)sizeof(BandRow) * 2 * N + r16(4 * N) + r16(real_bytes * 4 * N) + r16(4 * 2 * N);
    b += r16(real_bytes * 2 * S * 2 * N);
    if (field) b += r16(real_bytes * 2 * N) + r16(real_bytes * S * 2 * N);
    return b + 2 * buf_bytes;
}

int choose_band_shape(Plan *p, int64_t M, BandShape *out)
{
    const int N = p->N, bw = p->bandwidth;
    if (N > 256) return FTWA_ERR_UNSUPPORTED;
    const int real_bytes = p->precision == FTWA_FP64 ? 8 : 4;
    const int SZ = 2 * real_bytes, WC = SZ / 4;
    const int e_cap = kTmemColsPerWarp / (2 * WC);
    const int max_smem = 227 * 1024;
    const int sm = p->sm_count > 0 ? p->sm_count : 1;
    const int nblk = band_nblk(N), qoff = band_qoff(N);
    auto slices = [&](int sr) { return nblk - band_first_blk(sr % N, qoff); };
    for (int C = 1; C <= kMaxCluster; C *= 2) {
        if (p->cluster_override && C != p->cluster_override) continue;
        BandShape sh;
        sh.cluster = C;
        sh.qoff = qoff;
        // split spin-rows by their number of column-block slices
        double tot = 0;
        for (int sr = 0; sr < 2 * N; ++sr) tot += slices(sr);
        sh.row_begin[0] = 0;
        int sr = 0;
        double acc = 0;
        for (int r = 1; r < C; ++r) {
            const double target = tot * r / C;
            while (sr < 2 * N && acc + 0.5 * slices(sr) < target) {
                acc += slices(sr);
                ++sr;
            }
            sh.row_begin[r] = sr;
        }
        sh.row_begin[C] = 2 * N;
        int eps_max = 0;
        for (int r = 0; r < C; ++r) {
            int e = 0;
            for (int x = sh.row_begin[r]; x < sh.row_begin[r + 1]; ++x) e += band_row_len(N, bw, x);
            eps_max = std::max(eps_max, e);
        }
        int want = 1;
        if (C == 1) want = (int)std::max<long long>(1, std::min<long long>((M + sm - 1) / sm, 255));
        int best = 0;
        std::vector<std::vector<uint32_t>> best_items;
        int bestE = 0, bestK = 0;
        for (int S = 1; S <= want; ++S) {
            const int buf = ((S * eps_max * SZ + 15) / 16) * 16;
            if (band_smem(N, S, real_bytes, buf, p->drive || p->longrange || p->hop_drive) > max_smem) break;
            std::vector<std::vector<uint32_t>> its(C);
            int E = 0, K = 0;
            bool ok = true;
            for (int r = 0; r < C && ok; ++r) {
                // longest runs first; shorter runs pack the tensor-memory budget tighter
                bool placed = false;
                for (int R = 8; R >= 1 && !placed; R /= 2) {
                    int e, k;
                    placed = band_items(N, S, sh.row_begin[r], sh.row_begin[r + 1], e_cap, R, its[r], e, k);
                    if (placed) {
                        E = std::max(E, e);
                        K = std::max(K, k);
                    }
                }
                ok = placed;
            }
            if (!ok) break;
            best = S;
            best_items = its;
            bestE = E;
            bestK = K;
        }
        if (best == 0) continue;
        sh.slots = best;
        sh.E = bestE;
        sh.k_items = bestK;
        sh.items.assign((size_t)C * kWarps * bestK, 0xFFFFFFFFu);
        for (int r = 0; r < C; ++r) {
            // re-pack each rank's table to the common width bestK
            const int Kr = (int)(best_items[r].size() / kWarps);
            for (int w = 0; w < kWarps; ++w)
                for (int i = 0; i < Kr; ++i)
                    sh.items[((size_t)r * kWarps + w) * bestK + i] = best_items[r][(size_t)w * Kr + i];
        }
        sh.buf_bytes = ((best * eps_max * SZ + 15) / 16) * 16;
        sh.smem_bytes = std::max(kMinSmem, band_smem(N, best, real_bytes, sh.buf_bytes, p->drive || p->longrange || p->hop_drive));
        const long long batches = (M + best - 1) / best;
        sh.grid = (int)std::min<long long>(std::max<long long>(batches, 1), std::max(1, sm / C)) * C;
        *out = sh;
        return FTWA_OK;
    }
    return FTWA_ERR_UNSUPPORTED;
}

template <typename T, bool CLUSTER, bool UNIFORM_T, bool FIELD>
static int band_launch(Plan *p, BandShape &sh, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s)
{
    auto kern = band_stepper<T, CLUSTER, UNIFORM_T, FIELD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem_bytes);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(sh.grid, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = sh.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = sh.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = CLUSTER ? 1 : 0;
    if (CLUSTER) {
        int n_clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&n_clusters, kern, &cfg);
        if (e != cudaSuccess) return set_cuda_error(e);
        if (n_clusters < 1) return FTWA_ERR_UNSUPPORTED;
        sh.grid = std::min(sh.grid, n_clusters * sh.cluster);
        cfg.gridDim = dim3(sh.grid, 1, 1);
    }
    // upload the item table (plan-owned, reused while the shape is unchanged)
    const size_t bytes = sh.items.size() * sizeof(uint32_t);
    if (p->items_bytes < bytes) {
        cudaFree(p->d_items);
        p->d_items = nullptr;
        p->items_bytes = 0;
        e = cudaMalloc(&p->d_items, bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
        p->items_bytes = bytes;
    }
    if (p->items_host != sh.items) {
        // a changed table is uploaded (never during stream capture: batch
        // creation prepares every plan first)
        e = cudaMemcpyAsync(p->d_items, sh.items.data(), bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return set_cuda_error(e);
        p->items_host = sh.items;
    }
    p->shape.cluster = sh.cluster;
    p->shape.slots = sh.slots;
    p->shape.units_per_warp = sh.E;
    p->shape.smem_bytes = sh.smem_bytes;
    p->shape.grid = sh.grid;
    p->shape.variant = 1;
    p->shape.threads = kThreads;
    if (M == 0 || p->dry_run) return FTWA_OK;
    BandArgs<T> a{};
    a.nbr = p->d_nbr;
    a.tnb = std::is_same<T, double>::value ? reinterpret_cast<const T *>(p->d_t64)
                                           : reinterpret_cast<const T *>(p->d_t32);
    a.U = (T)p->U;
    a.dt = (T)p->dt;
    a.t_uniform = p->t_bond.empty() ? T(0) : (T)p->t_bond[0];
    a.N = p->N;
    a.bw = p->bandwidth;
    a.C = sh.cluster;
    a.S = sh.slots;
    a.E = sh.E;
    a.k_items = sh.k_items;
    a.buf_bytes = sh.buf_bytes;
    a.qoff = sh.qoff;
    const bool f64 = std::is_same<T, double>::value;
    a.amp = p->drive ? reinterpret_cast<const T *>(f64 ? (const void *)p->d_amp64 : (const void *)p->d_amp32) : nullptr;
    a.ftab = (p->drive || p->hop_drive) ? reinterpret_cast<const T *>(p->d_ftab) : nullptr;
    a.u = p->longrange ? reinterpret_cast<const T *>(f64 ? (const void *)p->d_u64 : (const void *)p->d_u32) : nullptr;
    for (int i = 0; i <= kMaxCluster; ++i) a.row_begin[i] = sh.row_begin[i];
    a.items = p->d_items;
    a.M = M;
    a.n_steps = n_steps;
    a.out_every = p->out_every;
    a.rho = reinterpret_cast<typename C2<T>::type *>(rho);
    a.snap = reinterpret_cast<T *>(snap);
    a.status = p->d_status;
    a.timeout_ns = p->timeout_ns;
    a.force_timeout = p->force_timeout;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    return set_cuda_error(e);
}

template <typename T, bool FIELD>
static int band_dispatch_d(Plan *p, BandShape &sh, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s)
{
    if (sh.cluster > 1)
        return p->uniform_t ? band_launch<T, true, true, FIELD>(p, sh, rho, M, n_steps, snap, s)
                            : band_launch<T, true, false, FIELD>(p, sh, rho, M, n_steps, snap, s);
    return p->uniform_t ? band_launch<T, false, true, FIELD>(p, sh, rho, M, n_steps, snap, s)
                        : band_launch<T, false, false, FIELD>(p, sh, rho, M, n_steps, snap, s);
}

template <typename T>
static int band_dispatch(Plan *p, BandShape &sh, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s)
{
    return (p->drive || p->longrange || p->hop_drive) ? band_dispatch_d<T, true>(p, sh, rho, M, n_steps, snap, s)
                                      : band_dispatch_d<T, false>(p, sh, rho, M, n_steps, snap, s);
}

// per RK4 stage time t = t_start + (step + c) dt, c = 0, 1/2, 1/2, 1 (in
// double): the on-site pulse f(t) (0 without a site drive) and the hopping
// scale m(t) = 1 + eps g(t) (1 without a hopping drive), interleaved
struct PulseArgs {
    double t0, sigma, omega, phase;
    int on;
};
__device__ __forceinline__ double pulse_at(const PulseArgs &q, double t)
{
    const double env = q.sigma > 0.0 ? exp(-(t - q.t0) * (t - q.t0) / (2.0 * q.sigma * q.sigma)) : 1.0;
    return env * cos(q.omega * (t - q.t0) + q.phase);
}
template <typename T>
__global__ void drive_table_kernel(T *ftab, long long n_steps, double t_start, double dt, PulseArgs site,
                                   PulseArgs hop, double hop_eps)
{
    const double c[4] = {0.0, 0.5, 0.5, 1.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 4 * n_steps;
         i += (long long)gridDim.x * blockDim.x) {
        const double t = t_start + ((double)(i / 4) + c[i % 4]) * dt;
        ftab[2 * i] = (T)(site.on ? pulse_at(site, t) : 0.0);
        ftab[2 * i + 1] = (T)(hop.on ? 1.0 + hop_eps * pulse_at(hop, t) : 1.0);
    }
}

static int prepare_drive(Plan *p, int64_t n_steps, double t_start, cudaStream_t s)
{
    const size_t bytes = (size_t)(p->precision == FTWA_FP64 ? 8 : 4) * 8 * (size_t)std::max<int64_t>(n_steps, 1);
    if (p->ftab_bytes < bytes) {
        cudaFree(p->d_ftab);
        p->d_ftab = nullptr;
        p->ftab_bytes = 0;
        cudaError_t e = cudaMalloc(&p->d_ftab, bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
        p->ftab_bytes = bytes;
    }
    if (n_steps == 0) return FTWA_OK;
    const long long n = 4 * n_steps;
    const int grid = (int)std::min<long long>((n + 255) / 256, 4096);
    const PulseArgs site{p->drive_t0, p->drive_sigma, p->drive_omega, p->drive_phase, p->drive ? 1 : 0};
    const PulseArgs hop{p->hop_t0, p->hop_sigma, p->hop_omega, p->hop_phase, p->hop_drive ? 1 : 0};
    if (p->precision == FTWA_FP64)
        drive_table_kernel<double><<<grid, 256, 0, s>>>(reinterpret_cast<double *>(p->d_ftab), n_steps, t_start,
                                                       p->dt, site, hop, p->hop_eps);
    else
        drive_table_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<float *>(p->d_ftab), n_steps, t_start,
                                                      p->dt, site, hop, p->hop_eps);
    return set_cuda_error(cudaGetLastError());
}

int launch_evolve(Plan *p, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s, double t_start)
{
    if (p->drive || p->longrange || p->hop_drive) {
        // the tabulated diagonal field (drive, long-range u) runs on the
        // banded stepper (both precisions)
        BandShape bs;
        int rc = choose_band_shape(p, M, &bs);
        if (rc != FTWA_OK) return rc;
        if ((p->drive || p->hop_drive) && M > 0 && !p->dry_run) {
            rc = prepare_drive(p, n_steps, t_start, s);
            if (rc != FTWA_OK) return rc;
        }
        return p->precision == FTWA_FP64 ? band_dispatch<double>(p, bs, rho, M, n_steps, snap, s)
                                         : band_dispatch<float>(p, bs, rho, M, n_steps, snap, s);
    }
    // automatic choice: the tiled stepper for FP32 (the banded one when no
    // tiled shape fits); for FP64 (DFMA-bound on this part) the packed-triangle
    // stepper, which does fewer flops per element
    if (p->variant_override == 3 || (p->variant_override == 0 && tile_supported(p))) {
        const int rc = launch_tile(p, rho, M, n_steps, snap, s);
        if (rc != FTWA_ERR_UNSUPPORTED || p->variant_override == 3) return rc;
    }
    const bool try_band = p->variant_override == 1 || (p->variant_override == 0 && p->precision == FTWA_FP32);
    if (try_band) {
        BandShape bs;
        if (choose_band_shape(p, M, &bs) == FTWA_OK)
            return p->precision == FTWA_FP64 ? band_dispatch<double>(p, bs, rho, M, n_steps, snap, s)
                                             : band_dispatch<float>(p, bs, rho, M, n_steps, snap, s);
        if (p->variant_override == 1) return FTWA_ERR_UNSUPPORTED;
    }
    StepperShape sh;
    int rc = choose_stepper_shape(p, M, &sh);
    if (rc != FTWA_OK) return rc;
    if (p->precision == FTWA_FP64)
        return sh.cluster > 1 ? dispatch_t<double, true>(p, sh, rho, M, n_steps, snap, s)
                              : dispatch_t<double, false>(p, sh, rho, M, n_steps, snap, s);
    return sh.cluster > 1 ? dispatch_t<float, true>(p, sh, rho, M, n_steps, snap, s)
                          : dispatch_t<float, false>(p, sh, rho, M, n_steps, snap, s);
}

}  // namespace ftwa
