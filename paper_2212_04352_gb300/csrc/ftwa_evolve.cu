// Persistent RK4 stepper for the fTWA equation of motion (Eq. 9).
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
//  - the diagonal Re rho_kk of both spins (the U coupling of Eq. 9) is
//    replicated into every CTA of the cluster at each stage.
// Work unit: 32 consecutive packed elements, one per lane.  A CTA owns a set
// of spin-rows (and, for small lattices, several samples, "slots").
//
// Per element (p, q), p <= q, spin s, the right-hand side of Eq. 9 is
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
    T U, dt;
    int N, C, S, E, meta_cols, buf_bytes;
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
    int pad[2];
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
__global__ void __launch_bounds__(kThreads, 1) rk4_stepper(const StepArgs<T> a)
{
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = a.N, S = a.S, C = a.C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = CLUSTER ? cluster_ctarank() : 0u;
    const uint32_t cid = CLUSTER ? cluster_id_x() : blockIdx.x;
    const uint32_t ncl = CLUSTER ? n_clusters_x() : gridDim.x;

    // ---- shared-memory carve-up ------------------------------------------
    SmemHeader *h = reinterpret_cast<SmemHeader *>(smem);
    int32_t *s_nbr = reinterpret_cast<int32_t *>(smem + 64);
    T *s_t = reinterpret_cast<T *>(smem + 64 + 4 * 256);
    uint32_t *s_row = reinterpret_cast<uint32_t *>(smem + 64 + 4 * 256 + sizeof(T) * 4 * 256);
    T *s_diag = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(s_row) +
                                      ((4 * S * 2 * N + 15) / 16) * 16);   // [2 buf][S][2N]
    unsigned char *bufA = reinterpret_cast<unsigned char *>(s_diag) + ((sizeof(T) * 2 * S * 2 * N + 15) / 16) * 16;
    const uint32_t bufA_s = smem_addr(bufA);
    const uint32_t diag_s = smem_addr(s_diag);
    const int diag_stride = S * 2 * N;   // elements per diag buffer

    const int rb0 = a.row_begin[rank], rb1 = a.row_begin[rank + 1];
    // elements per slot of this rank
    int eps = 0;
    for (int sr = rb0; sr < rb1; ++sr) eps += N - (sr % N);
    const int n_elem = eps * S;

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
    // shared::cluster address of element (p, p) of every spin-row, buffer A
    for (int idx = threadIdx.x; idx < S * 2 * N; idx += blockDim.x) {
        const int slot = idx / (2 * N), sr = idx % (2 * N);
        int owner = 0;
        while (owner + 1 < C && sr >= a.row_begin[owner + 1]) ++owner;
        int e_slot = 0, off = 0;
        for (int x = a.row_begin[owner]; x < a.row_begin[owner + 1]; ++x) {
            if (x < sr) off += N - (x % N);
            e_slot += N - (x % N);
        }
        const uint32_t local = bufA_s + (uint32_t)((slot * e_slot + off) * (int)sizeof(V));
        s_row[idx] = CLUSTER ? map_rank(local, owner) : local;
    }
    if (warp == 0) {
        tmem_alloc(smem_addr(&h->tmem_base), kTmemCols);
        tmem_relinquish();
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if constexpr (CLUSTER) cluster_sync_hw();   // barrier inits visible cluster-wide

    const uint32_t tbase = h->tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));
    constexpr int WC = sizeof(V) / 4;           // tensor-memory words per complex value
    const int E = a.E;
    const uint32_t t_meta = tbase, t_y0 = tbase + a.meta_cols, t_acc = tbase + a.meta_cols + E * WC;

    // ---- per-element metadata into tensor memory -----------------------------
    for (int j = 0; j < E; ++j) {
        const int e = (j * kWarps + warp) * 32 + lane;
        uint32_t meta = 0xFFFFFFFFu;
        if (e < n_elem) {
            const int slot = e / eps;
            int rem = e - slot * eps, sr = rb0;
            while (rem >= N - (sr % N)) {
                rem -= N - (sr % N);
                ++sr;
            }
            const int p = sr % N, q = p + rem, s = sr / N;
            meta = (uint32_t)q | ((uint32_t)p << 8) | ((uint32_t)s << 16) | ((uint32_t)slot << 17);
        }
        tmem_st1(t_meta + j, meta);
    }
    tmem_wait_st();

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
    const int twoN = 2 * N;
    const T half_dt = a.dt * T(0.5), sixth_dt = a.dt / T(6);

    for (long long b = cid; b < n_batches && h->abort == 0; b += ncl) {
        // ---- load rho(0) ---------------------------------------------------------
        for (int j = 0; j < E; ++j) {
            __syncwarp();
            const uint32_t meta = tmem_get1(t_meta + j);
            V v;
            v.x = T(0);
            v.y = T(0);
            if (meta != 0xFFFFFFFFu) {
                const int q = meta & 0xFF, p = (meta >> 8) & 0xFF, s = (meta >> 16) & 1, slot = meta >> 17;
                const long long m = b * S + slot;
                if (m < a.M) {
                    v = a.rho[((m * 2 + s) * N + p) * (long long)N + q];
                    if (p == q) {
                        v.y = T(0);
                        if (a.snap) a.snap[m * twoN + s * N + p] = v.x;
                    }
                }
                const int e = (j * kWarps + warp) * 32 + lane;
                sts2(bufA_s + (uint32_t)(e * (int)sizeof(V)), v);
                if (p == q) {
                    const uint32_t d = diag_s + (uint32_t)((slot * twoN + s * N + p) * (int)sizeof(T));
                    if constexpr (CLUSTER) {
                        for (int r = 0; r < C; ++r) stc1(map_rank(d, r), v.x);
                    } else {
                        s_diag[slot * twoN + s * N + p] = v.x;
                        (void)d;
                    }
                }
            }
            __syncwarp();
            tmem_put(t_y0 + j * WC, v);
        }
        tmem_wait_st();
        if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;

        // ---- RK4 steps -------------------------------------------------------------
        for (long long step = 0; step < a.n_steps && h->abort == 0; ++step) {
            const bool snap_now = a.snap && ((step + 1) % a.out_every == 0);
            const long long snap_row = (step + 1) / a.out_every;
            for (int stage = 0; stage < 4; ++stage) {
                const int cur = stage & 1;               // buffer read in this stage
                const uint32_t boff_cur = cur ? (uint32_t)a.buf_bytes : 0u;
                const uint32_t boff_nxt = cur ? 0u : (uint32_t)a.buf_bytes;
                const T *dg = s_diag + cur * diag_stride;
                for (int j = 0; j < E; ++j) {
                    __syncwarp();
                    const uint32_t meta = tmem_get1(t_meta + j);
                    V y0, acc;
                    tmem_get(t_y0 + j * WC, y0);
                    if (stage > 0) tmem_get(t_acc + j * WC, acc);
                    else acc = y0;
                    if (meta != 0xFFFFFFFFu) {
                        const int q = meta & 0xFF, p = (meta >> 8) & 0xFF, s = (meta >> 16) & 1, slot = meta >> 17;
                        const int e = (j * kWarps + warp) * 32 + lane;
                        const V own = lds2(bufA_s + boff_cur + (uint32_t)(e * (int)sizeof(V)), T());
                        const uint32_t *rows = s_row + slot * twoN + s * N;
                        const int nq = s_nbr[q], np = s_nbr[p];
                        T hr = T(0), hi = T(0);
                        // + sum_{k in nb(q)} t_qk rho_pk
#pragma unroll
                        for (int n = 0; n < 3; ++n) {
                            const int k = (nq >> (8 * n)) & 0xFF;
                            const T t = s_t[4 * q + n];
                            const bool fwd = k >= p;
                            const uint32_t ad =
                                rows[fwd ? p : k] + boff_cur + (uint32_t)((fwd ? k - p : p - k) * (int)sizeof(V));
                            const V v = CLUSTER ? ldc2(ad, T()) : lds2(ad, T());
                            hr = fma(t, v.x, hr);
                            hi = fma(t, fwd ? v.y : -v.y, hi);
                        }
                        // - sum_{k in nb(p)} t_pk rho_kq
#pragma unroll
                        for (int n = 0; n < 3; ++n) {
                            const int k = (np >> (8 * n)) & 0xFF;
                            const T t = s_t[4 * p + n];
                            const bool fwd = k <= q;
                            const uint32_t ad =
                                rows[fwd ? k : q] + boff_cur + (uint32_t)((fwd ? q - k : k - q) * (int)sizeof(V));
                            const V v = CLUSTER ? ldc2(ad, T()) : lds2(ad, T());
                            hr = fma(-t, v.x, hr);
                            hi = fma(-t, fwd ? v.y : -v.y, hi);
                        }
                        // + U (Re rho_pp,sbar - Re rho_qq,sbar) rho_pq
                        const T *db = dg + slot * twoN + (1 - s) * N;
                        const T g = a.U * (db[p] - db[q]);
                        hr = fma(g, own.x, hr);
                        hi = fma(g, own.y, hi);
                        // k = i (hr + i hi); on the diagonal Eq. 9 is real, so its
                        // imaginary part (pure rounding residue) is dropped
                        const T kx = -hi, ky = (p == q) ? T(0) : hr;
                        V nxt;
                        if (stage == 0) {
                            acc.x = kx;
                            acc.y = ky;
                            nxt.x = fma(half_dt, kx, y0.x);
                            nxt.y = fma(half_dt, ky, y0.y);
                        } else if (stage < 3) {
                            acc.x = fma(T(2), kx, acc.x);
                            acc.y = fma(T(2), ky, acc.y);
                            const T c = stage == 1 ? half_dt : a.dt;
                            nxt.x = fma(c, kx, y0.x);
                            nxt.y = fma(c, ky, y0.y);
                        } else {
                            nxt.x = fma(sixth_dt, acc.x + kx, y0.x);
                            nxt.y = fma(sixth_dt, acc.y + ky, y0.y);
                            y0 = nxt;
                        }
                        sts2(bufA_s + boff_nxt + (uint32_t)(e * (int)sizeof(V)), nxt);
                        if (p == q) {
                            const uint32_t d =
                                diag_s + (uint32_t)(((cur ^ 1) * diag_stride + slot * twoN + s * N + p) * (int)sizeof(T));
                            if constexpr (CLUSTER) {
                                for (int r = 0; r < C; ++r) stc1(map_rank(d, r), nxt.x);
                            } else {
                                s_diag[(cur ^ 1) * diag_stride + slot * twoN + s * N + p] = nxt.x;
                                (void)d;
                            }
                            if (stage == 3 && snap_now) {
                                const long long m = b * S + slot;
                                if (m < a.M) a.snap[(snap_row * a.M + m) * twoN + s * N + p] = nxt.x;
                            }
                        }
                    }
                    __syncwarp();
                    if (stage < 3) tmem_put(t_acc + j * WC, acc);
                    else tmem_put(t_y0 + j * WC, y0);
                }
                tmem_wait_st();
                if (!stage_barrier<CLUSTER>(h, phase, C, limit, a.status)) break;
            }
        }
        if (h->abort) break;

        // ---- write back rho(T) (full Hermitian matrix) ------------------------------
        for (int j = 0; j < E; ++j) {
            __syncwarp();
            const uint32_t meta = tmem_get1(t_meta + j);
            V y0;
            tmem_get(t_y0 + j * WC, y0);
            if (meta == 0xFFFFFFFFu) continue;
            const int q = meta & 0xFF, p = (meta >> 8) & 0xFF, s = (meta >> 16) & 1, slot = meta >> 17;
            const long long m = b * S + slot;
            if (m >= a.M) continue;
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
// Host side: launch-shape selection and launch.
// ---------------------------------------------------------------------------
static int smem_needed(int N, int S, int elem_bytes, int real_bytes, int buf_bytes)
{
    int b = 64 + 4 * 256 + real_bytes * 4 * 256;
    b += ((4 * S * 2 * N + 15) / 16) * 16;
    b += ((real_bytes * 2 * S * 2 * N + 15) / 16) * 16;
    b += 2 * buf_bytes;
    (void)elem_bytes;
    return b;
}

// Split the 2N spin-rows (row p of spin s has N - p packed elements) into C
// contiguous ranges with balanced element counts.
static void split_rows(int N, int C, int *rb)
{
    const long long total = (long long)N * (N + 1);
    rb[0] = 0;
    int sr = 0;
    long long acc = 0;
    for (int r = 1; r < C; ++r) {
        const long long target = total * r / C;
        while (sr < 2 * N && acc + (N - sr % N) / 2 < target) {
            acc += N - sr % N;
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
        split_rows(N, C, sh.row_begin);
        int eps_max = 0;
        for (int r = 0; r < C; ++r) {
            int eps = 0;
            for (int sr = sh.row_begin[r]; sr < sh.row_begin[r + 1]; ++sr) eps += N - sr % N;
            eps_max = std::max(eps_max, eps);
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
            const int units = (S * eps_max + 31) / 32;
            const int E = (units + kWarps - 1) / kWarps;
            const int meta_cols = ((E + 3) / 4) * 4;
            if (meta_cols + 2 * E * WC > 128) break;
            const int buf = ((S * eps_max * elem_bytes + 15) / 16) * 16;
            if (smem_needed(N, S, elem_bytes, real_bytes, buf) > max_smem) break;
            best = S;
        }
        if (best == 0) continue;
        sh.slots = best;
        const int units = (best * eps_max + 31) / 32;
        sh.units_per_warp = (units + kWarps - 1) / kWarps;
        sh.meta_cols = ((sh.units_per_warp + 3) / 4) * 4;
        sh.buf_bytes = ((best * eps_max * elem_bytes + 15) / 16) * 16;
        sh.smem_bytes = std::max(kMinSmem, smem_needed(N, best, elem_bytes, real_bytes, sh.buf_bytes));
        const long long batches = (M + best - 1) / best;
        const int max_groups = std::max(1, sm / C);
        sh.grid = (int)std::min<long long>(std::max<long long>(batches, 1), max_groups) * C;
        *out = sh;
        return FTWA_OK;
    }
    return FTWA_ERR_UNSUPPORTED;
}

template <typename T, bool CLUSTER>
static int launch_t(Plan *p, const StepperShape &sh, void *rho, int64_t M, int64_t n_steps, void *snap,
                    cudaStream_t s)
{
    StepArgs<T> a{};
    a.nbr = p->d_nbr;
    a.tnb = std::is_same<T, double>::value ? reinterpret_cast<const T *>(p->d_t64)
                                           : reinterpret_cast<const T *>(p->d_t32);
    a.U = (T)p->U;
    a.dt = (T)p->dt;
    a.N = p->N;
    a.C = sh.cluster;
    a.S = sh.slots;
    a.E = sh.units_per_warp;
    a.meta_cols = sh.meta_cols;
    a.buf_bytes = sh.buf_bytes;
    for (int i = 0; i <= kMaxCluster; ++i) a.row_begin[i] = sh.row_begin[i];
    a.M = M;
    a.n_steps = n_steps;
    a.out_every = p->out_every;
    a.rho = reinterpret_cast<typename C2<T>::type *>(rho);
    a.snap = reinterpret_cast<T *>(snap);
    a.status = p->d_status;
    a.timeout_ns = p->timeout_ns;
    a.force_timeout = p->force_timeout;
    auto kern = rk4_stepper<T, CLUSTER>;
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

int launch_evolve(Plan *p, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s)
{
    StepperShape sh;
    int rc = choose_stepper_shape(p, M, &sh);
    if (rc != FTWA_OK) return rc;
    if (sh.cluster > 1) {
        // clamp the grid to the clusters that can be co-resident
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
        cudaError_t e;
        if (p->precision == FTWA_FP64) {
            e = cudaFuncSetAttribute(rk4_stepper<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem_bytes);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n_clusters, rk4_stepper<double, true>, &cfg);
        } else {
            e = cudaFuncSetAttribute(rk4_stepper<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem_bytes);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n_clusters, rk4_stepper<float, true>, &cfg);
        }
        if (e != cudaSuccess) return set_cuda_error(e);
        if (n_clusters < 1) return FTWA_ERR_UNSUPPORTED;
        sh.grid = std::min(sh.grid, n_clusters * sh.cluster);
    }
    p->shape = sh;
    if (M == 0) return FTWA_OK;
    if (p->precision == FTWA_FP64)
        return sh.cluster > 1 ? launch_t<double, true>(p, sh, rho, M, n_steps, snap, s)
                              : launch_t<double, false>(p, sh, rho, M, n_steps, snap, s);
    return sh.cluster > 1 ? launch_t<float, true>(p, sh, rho, M, n_steps, snap, s)
                          : launch_t<float, false>(p, sh, rho, M, n_steps, snap, s);
}

}  // namespace ftwa
