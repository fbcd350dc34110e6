// Discrete adjoint of the RK4 integration of Eq. 6.
//
// Loss (linearised by the caller): L = sum_t sum_k g_t,k <n_k>(t), with
// <n_k>(t) = (1/M) sum_m Re rho^m_kk(t) + 1/2 (Eq. 5), so each sample's
// cotangent gets g_t,k / M on the diagonal at every output step.  With a
// correlation term sum_t sum_kl G_t,kl C_kl(t) (C the connected correlator
// of Eq. 5, C_kl = (1/M) sum_m x_mk x_ml - mu_k mu_l, x_mk = Re rho^m_kk),
// dC_kl/dx_mj = (1/M)[delta_jk (x_ml - mu_l) + delta_jl (x_mk - mu_k)], so
// sample m's diagonal entry j also gets (1/M) sum_l S_t,jl (x_ml - mu_t,l),
// S = G + G^T (symmetrised once per call into the plan's workspace).
//
// Per sample (one CTA): forward integration storing a checkpoint every
// ckpt_every steps; then, segment by segment backwards, the segment is
// replayed from its checkpoint (all its states kept), and each step is
// reversed stage by stage.  For y_{n+1} = y_n + h/6 (k1 + 2 k2 + 2 k3 + k4)
// with stage states Y1 = y_n, Y2 = y_n + h/2 k1, Y3 = y_n + h/2 k2,
// Y4 = y_n + h k3 and cotangent lam of y_{n+1}:
//   G4 = h/6 lam;  w4 = VJP(Y4)[G4];  G3 = h/3 lam + h w4
//   w3 = VJP(Y3)[G3];  G2 = h/3 lam + h/2 w3
//   w2 = VJP(Y2)[G2];  G1 = h/6 lam + h/2 w2
//   w1 = VJP(Y1)[G1];  lam_n = lam + w1 + w2 + w3 + w4
// Under the real inner product <A, B> = Re tr(A^dagger B):
//   VJP_f(Y)[v] = -f_D(v)  with D = diag(Re Y_kk,sbar + 1/2) held fixed, plus
//   the coupling of f's U term to the other spin's diagonal,
//   (w_sbar)_kk += c_k = -2U sum_j Im(conj(v_kj) Y_kj)  (full row k of spin s);
//   dL/dU    += sum_ij (d_i - d_j)(-Im(conj(v_ij) Y_ij));
//   dL/dt_b  += sum over elements (i, j) of -Im(conj(v_ij) Y_ik) for the
//               row-part neighbours k of j (bond (j, k)) and
//               +Im(conj(v_ij) Y_kj) for the column-part neighbours k of i
//               (bond (i, k)).
// Sums over all ordered (i, j) are taken over the stored upper triangle with
// weight 2 off the diagonal and 1 on it (v and Y are Hermitian).  Finally
// rho_ii(0) = n_i - 1/2 and rho_ij(0) = xi_ij s_ij(n) (Eq. 7) give
//   dL/dn_i += Re lam_ii(0) + sum_{j != i} Re(conj(lam_ij) xi_ij) (1 - 2 n_j)/(2 s_ij)
// (pairs with s_ij = 0 are skipped: the map n -> s is not differentiable there).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "ftwa_internal.h"

namespace ftwa {

namespace adj {

template <typename T> struct C2T;
template <> struct C2T<float> { using type = float2; };
template <> struct C2T<double> { using type = double2; };

// Launch shapes: the per-sample work is a sequence of dependent passes over
// the sample's matrices in a per-CTA workspace (L2-resident when few enough
// samples are in flight).  FP32 runs one 1024-thread CTA per SM, FP64 four
// 256-thread CTAs (see launch_adjoint_t).  (Staging each evaluation's input
// in shared memory, one sample per SM, measured slower.)

template <typename T>
struct AdjArgs {
    int N, B, NE;                 // sites, bonds, packed elements (both spins)
    const int32_t *nbr;           // [N] packed slots
    const int32_t *nbr_bond;      // [N][3] bond of each slot (-1 if none)
    const int32_t *bonds;         // [B][2] bond endpoints
    const T *tnb;                 // [N][4]
    const double *nocc;           // [2][N] initial occupations
    T U, dt;
    int out_every, ckpt_every;
    long long n_steps, M;
    unsigned long long seed;
    const double *dL;             // [n_out][2N] or null
    const double *dS;             // [n_out][2N][2N] S = G + G^T of a correlation term, or null
    const double *mu;             // [n_out][2N] sample means of Re rho_kk (with dS)
    double *gU, *gt, *gn;         // outputs (accumulated with atomics)
    typename C2T<T>::type *ws;    // per-CTA workspace
    long long ws_stride;          // elements per CTA
    int *status;
};

// packed index of (s, a, b), a <= b
__device__ __forceinline__ int pidx(int N, int s, int a, int b)
{
    return s * (N * (N + 1) / 2) + a * N - a * (a - 1) / 2 + (b - a);
}

template <typename V>
__device__ __forceinline__ V getc(const V *buf, int N, int s, int a, int b)
{
    if (a <= b) return buf[pidx(N, s, a, b)];
    V v = buf[pidx(N, s, b, a)];
    v.y = -v.y;
    return v;
}

// Philox4x32-10 and the Box-Muller normal of Eq. 7 (same counter layout as
// the sampler: key (seed_lo, seed_hi), counter (m_lo, m_hi, s, p))
__device__ __forceinline__ double2 xi_of(unsigned long long seed, long long m, int s, uint32_t p)
{
    uint32_t c0 = (uint32_t)m, c1 = (uint32_t)((unsigned long long)m >> 32), c2 = (uint32_t)s, c3 = p;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const unsigned long long b1 = ((unsigned long long)c1 << 32) | c0;
    const unsigned long long b2 = ((unsigned long long)c3 << 32) | c2;
    const double u1 = (double)(b1 >> 11) * 0x1p-53 + 0x1p-54;
    const double u2 = (double)(b2 >> 11) * 0x1p-53 + 0x1p-54;
    const double r = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    return make_double2(r * cs, r * sn);
}

template <typename T>
struct Smem {
    uint32_t *elem;     // [NE]: a | b << 8 | s << 16
    int32_t *nbr;       // [N]
    int32_t *bond;      // [N][3]
    int32_t *bxy;       // [B][2]
    T *cacc;            // [2][N] diagonal coupling sums of one VJP
    T *bacc;            // [B] bond sums of one VJP
    T *wd;              // [2][N] diagonal of W before the coupling
    double *gt;         // [B]
    double *gn;         // [2][N]
    double *xc;         // [2N] centred diagonal of the sample at an output step
};

// One RK4 stage pass on the packed upper triangle, k = f(src) (Eq. 6)
// combined in the same pass (no separate k buffer):
//   MODE 0: out = y0 + c k              (stage states of the reverse sweep)
//   MODE 1: acc = k;      out = y0 + c k
//   MODE 2: acc += 2 k;   out = y0 + c k
//   MODE 3: out = y0 + c (acc + k)      (c = h/6: the step's result)
// out must not alias src (other threads gather src).  With lam != nullptr
// the pass also starts the reverse step's cotangents: g4 = h/6 lam,
// lam_new = lam.  Ends with a CTA barrier.
template <int MODE, typename T>
__device__ void f_pass(const AdjArgs<T> &a, const Smem<T> &sm, const typename C2T<T>::type *src,
                       const typename C2T<T>::type *y0, typename C2T<T>::type *acc, typename C2T<T>::type *out,
                       T c, const typename C2T<T>::type *lam = nullptr, typename C2T<T>::type *g4 = nullptr,
                       typename C2T<T>::type *lam_new = nullptr)
{
    using V = typename C2T<T>::type;
    const int N = a.N;
    const T h6 = a.dt / T(6);
    for (int e = threadIdx.x; e < a.NE; e += blockDim.x) {
        const uint32_t d = sm.elem[e];
        const int i = d & 0xFF, j = (d >> 8) & 0xFF, s = d >> 16;
        const int nj = sm.nbr[j], ni = sm.nbr[i];
        T hr = T(0), hi = T(0);
        // all three slots: an empty slot has t = 0 and a valid column
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            const V v = getc(src, N, s, i, (nj >> (8 * n)) & 0xFF);
            const T t = a.tnb[4 * j + n];
            hr = fma(t, v.x, hr);
            hi = fma(t, v.y, hi);
        }
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            const V v = getc(src, N, s, (ni >> (8 * n)) & 0xFF, j);
            const T t = a.tnb[4 * i + n];
            hr = fma(-t, v.x, hr);
            hi = fma(-t, v.y, hi);
        }
        const V own = src[e];
        const T g = a.U * (src[pidx(N, 1 - s, i, i)].x - src[pidx(N, 1 - s, j, j)].x);
        hr = fma(g, own.x, hr);
        hi = fma(g, own.y, hi);
        V k;
        k.x = -hi;
        k.y = (i == j) ? T(0) : hr;
        const V b = y0[e];
        V o;
        if constexpr (MODE == 3) {
            const V q = acc[e];
            o.x = fma(c, q.x + k.x, b.x);
            o.y = fma(c, q.y + k.y, b.y);
        } else {
            if constexpr (MODE == 1) acc[e] = k;
            if constexpr (MODE == 2) {
                V q = acc[e];
                q.x = fma(T(2), k.x, q.x);
                q.y = fma(T(2), k.y, q.y);
                acc[e] = q;
            }
            o.x = fma(c, k.x, b.x);
            o.y = fma(c, k.y, b.y);
        }
        out[e] = o;
        if (lam) {
            const V l = lam[e];
            V q;
            q.x = h6 * l.x;
            q.y = h6 * l.y;
            g4[e] = q;
            lam_new[e] = l;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cotangent bookkeeping of one reversed RK4 stage for element e with
// W = VJP(Y_s)[G_s]: lam_new += W and the next stage's G = ca lam + cb W, or,
// for the first stage (last = true), lam = lam_new + W.
template <typename V, typename T>
__device__ __forceinline__ void cot_update(int e, V o, V *gout, V *lam, V *lam_new, T ca, T cb, bool last)
{
    V ln = lam_new[e];
    ln.x += o.x;
    ln.y += o.y;
    if (last) {
        lam[e] = ln;
    } else {
        lam_new[e] = ln;
        const V l = lam[e];
        V g;
        g.x = fma(cb, o.x, ca * l.x);
        g.y = fma(cb, o.y, ca * l.y);
        gout[e] = g;
    }
}

// W = VJP_f(Y)[v] for FP32 plans, with the cotangent update of the stage
// (cot_update) fused; accumulates dL/dU (register) and dL/dt_b (shared
// memory), in one pass over the stored upper triangle, a warp per row (coalesced):
//  - elementwise: w = -f_D(v) with D from Y, and the U gradient;
//  - the U term's coupling to the other spin's diagonal,
//      c_k = -2U sum_j P_kj,  P_kj = Im(conj(v_kj) Y_kj)   (full row k);
//    P is antisymmetric for Hermitian v, Y (P_jk = -P_kj), so a stored
//    element (i, j), i < j, adds P_ij to c_i and -P_ij to c_j;
//  - the hopping gradient of bond b = (x, y): with Hermitian v and Y,
//      <v, d f / d t_b> = -2 Im[(v Y)_xy + (v Y)_yx],
//    (v Y)_pk = sum_q v_pq conj(Y_kq) for k in nb(p).  The ordered pair
//    (p, q) = (i, j) of a stored element gives Im(v_ij conj(Y_kj)), k in
//    nb(i) (the column-part neighbours of Eq. 6), to the bond (i, k); the
//    mirrored pair (p, q) = (j, i), i < j, gives Im(conj(v_ij) Y_ik), k in
//    nb(j) (the row-part neighbours), to the bond (j, k).
// Row-fixed sums (c_i, bonds of row i) are reduced over the warp once per
// row; column-dependent ones (c_j, bonds of column j) are added per lane to
// shared memory (distinct columns per lane: little contention).
template <typename T>
__device__ void vjp_rows(const AdjArgs<T> &a, const Smem<T> &sm, const typename C2T<T>::type *Y,
                         const typename C2T<T>::type *v, typename C2T<T>::type *gout, typename C2T<T>::type *lam,
                         typename C2T<T>::type *lam_new, T ca, T cb, bool last, double &gU)
{
    using V = typename C2T<T>::type;
    const int N = a.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) sm.cacc[i] = T(0);
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) sm.bacc[b] = T(0);
    __syncthreads();
    for (int r = warp; r < 2 * N; r += n_warps) {
        const int s = r / N, i = r % N;
        const int ni = sm.nbr[i], degi = (ni >> 24) & 0xFF;
        const int e0 = pidx(N, s, i, i);
        const T di = Y[pidx(N, 1 - s, i, i)].x;
        T ci = T(0), gu = T(0), bi[3] = {T(0), T(0), T(0)};
        for (int j = i + lane; j < N; j += 32) {
            const int e = e0 + (j - i);
            const int nj = sm.nbr[j], degj = (nj >> 24) & 0xFF;
            const V vo = v[e], yo = Y[e];
            T hr = T(0), hi = T(0);
            // row part: neighbours k of j (all three slots: an empty slot has
            // t = 0 and a valid column, so the loads are unconditional)
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                const int k = (nj >> (8 * n)) & 0xFF;
                const V vk = getc(v, N, s, i, k);
                const T t = a.tnb[4 * j + n];
                hr = fma(t, vk.x, hr);
                hi = fma(t, vk.y, hi);
                if (i != j && n < degj) {
                    // Im(conj(v_ij) Y_ik) -> bond (j, k)
                    const V yk = getc(Y, N, s, i, k);
                    atomicAdd(&sm.bacc[sm.bond[3 * j + n]], vo.x * yk.y - vo.y * yk.x);
                }
            }
            // column part: neighbours k of i (empty slots accumulate into bi[n]
            // but are never flushed)
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                const int k = (ni >> (8 * n)) & 0xFF;
                const V vk = getc(v, N, s, k, j);
                const T t = a.tnb[4 * i + n];
                hr = fma(-t, vk.x, hr);
                hi = fma(-t, vk.y, hi);
                // Im(v_ij conj(Y_kj)) -> bond (i, k)
                const V yk = getc(Y, N, s, k, j);
                bi[n] += vo.y * yk.x - vo.x * yk.y;
            }
            const T dj = Y[pidx(N, 1 - s, j, j)].x;
            const T g = a.U * (di - dj);
            hr = fma(g, vo.x, hr);
            hi = fma(g, vo.y, hi);
            // w = -i (hr + i hi) = (hi, -hr)
            V o;
            o.x = hi;
            o.y = -hr;
            if (i != j) {
                const T P = vo.x * yo.y - vo.y * yo.x;   // Im(conj(v_ij) Y_ij)
                gu = fma(di - dj, P, gu);
                ci += P;
                atomicAdd(&sm.cacc[s * N + j], -P);
                cot_update(e, o, gout, lam, lam_new, ca, cb, last);
            } else {
                sm.wd[s * N + i] = hi;   // the coupling is added once all rows are done
            }
        }
        // dL/dU: weight 2, the stored (i, j) stands for (i, j) and (j, i); the
        // row's sum is taken in T (no FP64 work per element in FP32 plans)
        gU += -2.0 * (double)gu;
        for (int o = 16; o > 0; o >>= 1) {
            ci += __shfl_xor_sync(0xffffffffu, ci, o);
#pragma unroll
            for (int n = 0; n < 3; ++n) bi[n] += __shfl_xor_sync(0xffffffffu, bi[n], o);
        }
        if (lane == 0) {
            atomicAdd(&sm.cacc[s * N + i], ci);
            for (int n = 0; n < degi; ++n) atomicAdd(&sm.bacc[sm.bond[3 * i + n]], bi[n]);
        }
    }
    __syncthreads();
    // diagonal elements: w_kk,s plus the coupling c of row (sbar, k); bond
    // sums into the CTA's totals
    for (int e = threadIdx.x; e < 2 * N; e += blockDim.x) {
        const int s = e / N, k = e % N;
        V o;
        o.x = sm.wd[e] + (T)(-2.0 * (double)a.U * (double)sm.cacc[(1 - s) * N + k]);
        o.y = T(0);
        cot_update(pidx(N, s, k, k), o, gout, lam, lam_new, ca, cb, last);
    }
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) sm.gt[b] += -2.0 * (double)sm.bacc[b];
    __syncthreads();
}

// w = VJP_f(Y)[v] for FP64 plans (the same sums as vjp_rows, taken as dot
// products): accumulates dL/dU (register) and dL/dt_b (shared memory).
//  - elementwise: w = -f_D(v) with D from Y, and the U gradient;
//  - the U term's coupling to the other spin's diagonal,
//      c_k = -2U sum_j Im(conj(v_kj) Y_kj)   (full row k), one warp per row;
//  - the hopping gradient of bond b = (x, y): with Hermitian v and Y,
//      <v, d f / d t_b> = -2 Im[(v Y)_xy + (v Y)_yx]   (per spin),
//    dot products over the full rows/columns, one warp per bond.
// Every shared-memory sum has one writer: no atomics (measured faster than
// vjp_rows for FP64, whose shared-memory atomics on doubles are slow).
template <typename T>
__device__ void vjp_dot(const AdjArgs<T> &a, const Smem<T> &sm, const typename C2T<T>::type *Y,
                    const typename C2T<T>::type *v, typename C2T<T>::type *w, double &gU)
{
    using V = typename C2T<T>::type;
    const int N = a.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (int e = threadIdx.x; e < a.NE; e += blockDim.x) {
        const uint32_t d = sm.elem[e];
        const int i = d & 0xFF, j = (d >> 8) & 0xFF, s = d >> 16;
        const int nj = sm.nbr[j], ni = sm.nbr[i];
        const V vo = v[e], yo = Y[e];
        T hr = T(0), hi = T(0);
        // row part: neighbours k of j
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            const V vk = getc(v, N, s, i, (nj >> (8 * n)) & 0xFF);
            const T t = a.tnb[4 * j + n];
            hr = fma(t, vk.x, hr);
            hi = fma(t, vk.y, hi);
        }
        // column part: neighbours k of i
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            const V vk = getc(v, N, s, (ni >> (8 * n)) & 0xFF, j);
            const T t = a.tnb[4 * i + n];
            hr = fma(-t, vk.x, hr);
            hi = fma(-t, vk.y, hi);
        }
        const T di = Y[pidx(N, 1 - s, i, i)].x, dj = Y[pidx(N, 1 - s, j, j)].x;
        const T g = a.U * (di - dj);
        hr = fma(g, vo.x, hr);
        hi = fma(g, vo.y, hi);
        // w = -i (hr + i hi) = (hi, -hr)
        V o;
        o.x = hi;
        o.y = (i == j) ? T(0) : -hr;
        w[e] = o;
        if (i != j) {
            // weight 2: the stored (i, j) stands for (i, j) and (j, i)
            const double P = (double)vo.x * yo.y - (double)vo.y * yo.x;   // Im(conj(v_ij) Y_ij)
            gU += 2.0 * (double)(di - dj) * (-P);
        }
    }
    for (int r = warp; r < 2 * N; r += n_warps) {
        const int s = r / N, k = r % N;
        double acc = 0.0;
        for (int j = lane; j < N; j += 32) {
            const V vk = getc(v, N, s, k, j), yk = getc(Y, N, s, k, j);
            acc += (double)vk.x * yk.y - (double)vk.y * yk.x;
        }
        acc = warp_sum(acc);
        if (lane == 0) sm.cacc[r] = (T)(-2.0 * (double)a.U * acc);
    }
    for (int b = warp; b < a.B; b += n_warps) {
        const int x = sm.bxy[2 * b], y = sm.bxy[2 * b + 1];
        double acc = 0.0;
        for (int s = 0; s < 2; ++s)
            for (int i = lane; i < N; i += 32) {
                // Im(v_xi Y_iy) + Im(v_yi Y_ix)
                const V v1 = getc(v, N, s, x, i), y1 = getc(Y, N, s, i, y);
                const V v2 = getc(v, N, s, y, i), y2 = getc(Y, N, s, i, x);
                acc += (double)v1.x * y1.y + (double)v1.y * y1.x + (double)v2.x * y2.y + (double)v2.y * y2.x;
            }
        acc = warp_sum(acc);
        if (lane == 0) sm.gt[b] += -2.0 * acc;
    }
    __syncthreads();
    // coupling to the other spin's diagonal
    for (int e = threadIdx.x; e < 2 * N; e += blockDim.x) {
        const int s = e / N, k = e % N;
        V &x = w[pidx(N, 1 - s, k, k)];
        x.x += sm.cacc[e];
    }
    __syncthreads();
}

// one RK4 step y1 = y0 + h/6 (k1 + 2 k2 + 2 k3 + k4) in four fused passes
// (ys, ys2: stage states; acc: the weighted sum of the k's)
template <typename T>
__device__ void rk4(const AdjArgs<T> &a, const Smem<T> &sm, const typename C2T<T>::type *y0,
                    typename C2T<T>::type *y1, typename C2T<T>::type *ys, typename C2T<T>::type *ys2,
                    typename C2T<T>::type *acc)
{
    const T h = a.dt;
    f_pass<1>(a, sm, y0, y0, acc, ys, h * T(0.5));
    f_pass<2>(a, sm, ys, y0, acc, ys2, h * T(0.5));
    f_pass<2>(a, sm, ys2, y0, acc, ys, h);
    f_pass<3>(a, sm, ys, y0, acc, y1, h / T(6));
}

template <typename T, int THREADS, int CTAS>
__global__ void __launch_bounds__(THREADS, CTAS) adjoint_kernel(const AdjArgs<T> a)
{
    using V = typename C2T<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = a.N, NE = a.NE;
    Smem<T> sm;
    unsigned char *p = smem;
    sm.cacc = reinterpret_cast<T *>(p);
    p += sizeof(double) * 2 * N;
    sm.bacc = reinterpret_cast<T *>(p);
    p += sizeof(double) * std::max(a.B, 1);
    sm.wd = reinterpret_cast<T *>(p);
    p += sizeof(double) * 2 * N;
    sm.gt = reinterpret_cast<double *>(p);
    p += sizeof(double) * std::max(a.B, 1);
    sm.gn = reinterpret_cast<double *>(p);
    p += sizeof(double) * 2 * N;
    sm.xc = reinterpret_cast<double *>(p);
    p += sizeof(double) * 2 * N;
    sm.nbr = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * N;
    sm.bond = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * 3 * N;
    sm.bxy = reinterpret_cast<int32_t *>(p);
    p += sizeof(int32_t) * 2 * std::max(a.B, 1);
    sm.elem = reinterpret_cast<uint32_t *>(p);

    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        sm.nbr[i] = a.nbr[i];
        for (int n = 0; n < 3; ++n) sm.bond[3 * i + n] = a.nbr_bond[3 * i + n];
    }
    for (int i = threadIdx.x; i < a.B; i += blockDim.x) {
        sm.gt[i] = 0.0;
        sm.bxy[2 * i] = a.bonds[2 * i];
        sm.bxy[2 * i + 1] = a.bonds[2 * i + 1];
    }
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) sm.gn[i] = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < N; ++i)
            for (int j = i + threadIdx.x; j < N; j += blockDim.x) sm.elem[pidx(N, s, i, j)] = i | (j << 8) | (s << 16);
    __syncthreads();

    const int n_seg = (int)(a.n_steps / a.ckpt_every);
    V *ws = a.ws + (long long)blockIdx.x * a.ws_stride;
    V *ckpt = ws;                                         // [n_seg][NE]
    V *seg = ckpt + (long long)n_seg * NE;                // [ckpt_every + 1][NE]
    V *Y2 = seg + (long long)(a.ckpt_every + 1) * NE;
    V *Y3 = Y2 + NE, *Y4 = Y3 + NE, *A = Y4 + NE, *lam = A + NE, *G = lam + NE, *W = G + NE,
      *lam_new = W + NE, *cur = lam_new + NE, *nxt = cur + NE;
    const T h = a.dt;
    const int twoN = 2 * N;
    const double invM = 1.0 / (double)a.M;
    double gU = 0.0;

    for (long long m = blockIdx.x; m < a.M; m += gridDim.x) {
        // ---- rho(0) of sample m (Eq. 7) --------------------------------------
        for (int e = threadIdx.x; e < NE; e += blockDim.x) {
            const uint32_t d = sm.elem[e];
            const int i = d & 0xFF, j = (d >> 8) & 0xFF, s = d >> 16;
            const double ni = a.nocc[s * N + i], nj = a.nocc[s * N + j];
            V v;
            if (i == j) {
                v.x = (T)(ni - 0.5);
                v.y = T(0);
            } else {
                const double var = 0.5 * (ni + nj - 2.0 * ni * nj);
                const double sd = var > 0.0 ? sqrt(var) : 0.0;
                const double2 x = xi_of(a.seed, m, s, (uint32_t)(i * N - i * (i + 1) / 2 + (j - i - 1)));
                v.x = (T)(x.x * sd);
                v.y = (T)(x.y * sd);
            }
            cur[e] = v;
        }
        __syncthreads();
        // ---- forward with checkpoints ------------------------------------------
        for (long long step = 0; step < a.n_steps; ++step) {
            if (step % a.ckpt_every == 0) {
                V *c = ckpt + (step / a.ckpt_every) * NE;
                for (int e = threadIdx.x; e < NE; e += blockDim.x) c[e] = cur[e];
                __syncthreads();
            }
            rk4(a, sm, cur, nxt, Y2, Y3, A);
            V *t = cur;
            cur = nxt;
            nxt = t;
        }
        // ---- cotangent at the final step --------------------------------------------
        for (int e = threadIdx.x; e < NE; e += blockDim.x) {
            lam[e].x = T(0);
            lam[e].y = T(0);
        }
        __syncthreads();
        // cotangent of the loss at output step `step`; y is the sample's state there
        auto inject = [&](long long step, const V *y) {
            if (step % a.out_every) return;
            const long long t = step / a.out_every;
            if (a.dS) {
                for (int e = threadIdx.x; e < twoN; e += blockDim.x) {
                    const int s = e / N, k = e % N;
                    sm.xc[e] = (double)y[pidx(N, s, k, k)].x - a.mu[t * twoN + e];
                }
                __syncthreads();
                // (1/M) sum_l S_jl x_l: a warp per row j, lanes over l
                const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
                const double *S = a.dS + t * (long long)twoN * twoN;
                for (int j = threadIdx.x >> 5; j < twoN; j += nw) {
                    double acc = 0.0;
                    for (int l = lane; l < twoN; l += 32) acc = fma(S[(long long)j * twoN + l], sm.xc[l], acc);
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) {
                        const double gj = a.dL ? a.dL[t * twoN + j] : 0.0;
                        const int s = j / N, k = j % N;
                        lam[pidx(N, s, k, k)].x += (T)((gj + acc) * invM);
                    }
                }
            } else {
                const double *g = a.dL + t * twoN;
                for (int e = threadIdx.x; e < twoN; e += blockDim.x) {
                    const int s = e / N, k = e % N;
                    lam[pidx(N, s, k, k)].x += (T)(g[e] * invM);
                }
            }
            __syncthreads();
        };
        inject(a.n_steps, cur);
        // ---- reverse sweep ----------------------------------------------------------
        for (int sg = n_seg - 1; sg >= 0; --sg) {
            for (int e = threadIdx.x; e < NE; e += blockDim.x) seg[e] = ckpt[(long long)sg * NE + e];
            __syncthreads();
            // states 1 .. ckpt_every-1 of the segment (the reverse sweep never
            // reads the last one)
            for (int r = 0; r + 1 < a.ckpt_every; ++r)
                rk4(a, sm, seg + (long long)r * NE, seg + (long long)(r + 1) * NE, Y2, Y3, A);
            for (int r = a.ckpt_every - 1; r >= 0; --r) {
                const V *y = seg + (long long)r * NE;
                // stage states Y2..Y4 (and G = h/6 lam, lam_new = lam)
                f_pass<0>(a, sm, y, y, (V *)nullptr, Y2, h * T(0.5), lam, G, lam_new);
                f_pass<0>(a, sm, Y2, y, (V *)nullptr, Y3, h * T(0.5));
                f_pass<0>(a, sm, Y3, y, (V *)nullptr, Y4, h);
                if constexpr (std::is_same<T, float>::value) {
                    // stage cotangents alternate between G and W
                    vjp_rows(a, sm, Y4, G, W, lam, lam_new, h / T(3), h, false, gU);
                    vjp_rows(a, sm, Y3, W, G, lam, lam_new, h / T(3), h * T(0.5), false, gU);
                    vjp_rows(a, sm, Y2, G, W, lam, lam_new, h / T(6), h * T(0.5), false, gU);
                    vjp_rows(a, sm, y, W, (V *)nullptr, lam, lam_new, T(0), T(0), true, gU);
                } else {
                    vjp_dot(a, sm, Y4, G, W, gU);
                    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
                        lam_new[e].x += W[e].x;
                        lam_new[e].y += W[e].y;
                        G[e].x = fma(h, W[e].x, h / T(3) * lam[e].x);
                        G[e].y = fma(h, W[e].y, h / T(3) * lam[e].y);
                    }
                    __syncthreads();
                    vjp_dot(a, sm, Y3, G, W, gU);
                    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
                        lam_new[e].x += W[e].x;
                        lam_new[e].y += W[e].y;
                        G[e].x = fma(h * T(0.5), W[e].x, h / T(3) * lam[e].x);
                        G[e].y = fma(h * T(0.5), W[e].y, h / T(3) * lam[e].y);
                    }
                    __syncthreads();
                    vjp_dot(a, sm, Y2, G, W, gU);
                    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
                        lam_new[e].x += W[e].x;
                        lam_new[e].y += W[e].y;
                        G[e].x = fma(h * T(0.5), W[e].x, h / T(6) * lam[e].x);
                        G[e].y = fma(h * T(0.5), W[e].y, h / T(6) * lam[e].y);
                    }
                    __syncthreads();
                    vjp_dot(a, sm, y, G, W, gU);
                    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
                        lam[e].x = lam_new[e].x + W[e].x;
                        lam[e].y = lam_new[e].y + W[e].y;
                    }
                    __syncthreads();
                }
                inject((long long)sg * a.ckpt_every + r, y);
            }
        }
        // ---- initial occupations -------------------------------------------------------
        for (int e = threadIdx.x; e < NE; e += blockDim.x) {
            const uint32_t d = sm.elem[e];
            const int i = d & 0xFF, j = (d >> 8) & 0xFF, s = d >> 16;
            if (i == j) {
                atomicAdd(&sm.gn[s * N + i], (double)lam[e].x);
            } else {
                const double ni = a.nocc[s * N + i], nj = a.nocc[s * N + j];
                const double var = 0.5 * (ni + nj - 2.0 * ni * nj);
                if (var > 0.0) {
                    const double sd = sqrt(var);
                    const double2 x = xi_of(a.seed, m, s, (uint32_t)(i * N - i * (i + 1) / 2 + (j - i - 1)));
                    const double re = (double)lam[e].x * x.x + (double)lam[e].y * x.y;   // Re(conj(lam) xi)
                    atomicAdd(&sm.gn[s * N + i], re * (1.0 - 2.0 * nj) / (2.0 * sd));
                    atomicAdd(&sm.gn[s * N + j], re * (1.0 - 2.0 * ni) / (2.0 * sd));
                }
            }
        }
        __syncthreads();
    }
    // ---- publish this CTA's sums -------------------------------------------------
    __shared__ double red[THREADS / 32];
    double v = gU;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
        if (a.gU) atomicAdd(a.gU, t);
    }
    for (int i = threadIdx.x; i < a.B; i += blockDim.x)
        if (a.gt) atomicAdd(&a.gt[i], sm.gt[i]);
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x)
        if (a.gn) atomicAdd(&a.gn[i], sm.gn[i]);
}

__global__ void zero_kernel(double *x, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

// S_t = G_t + G_t^T and mu_t = <n>_t - 1/2 of a correlation term ([T][K][K], [T][K])
__global__ void symmetrise_kernel(const double *G, const double *occ, int T, int K, double *S, double *mu)
{
    const long long n = (long long)T * K * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / ((long long)K * K);
        const int k = (int)((i / K) % K), l = (int)(i % K);
        S[i] = G[i] + G[(t * K + l) * K + k];
        if (l == 0) mu[t * K + k] = occ[t * K + k] - 0.5;
    }
}

}  // namespace adj

template <typename T>
static int launch_adjoint_t(Plan *p, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every, const double *dL,
                            const double *dS, const double *mu, double *gU, double *gt, double *gn, cudaStream_t s)
{
    using namespace adj;
    using V = typename C2T<T>::type;
    const int N = p->N;
    const int NE = N * (N + 1);
    const int n_seg = (int)(n_steps / ckpt_every);
    const long long stride = (long long)(n_seg + ckpt_every + 1 + 11) * NE;
    const int smem_tables = (int)(sizeof(double) * (8 * N + 2 * std::max(p->B, 1)) + sizeof(int32_t) * 4 * N +
                                  sizeof(int32_t) * 2 * std::max(p->B, 1) + sizeof(uint32_t) * NE + 64);
    // FP32: one 1024-thread CTA per SM, so that the samples in flight keep
    // their working sets in L2 (measured 1.4x faster than four 256-thread
    // CTAs, and faster than 768 threads with more registers each); FP64 is
    // bound by the FP64 pipe either way
    const int ctas = std::is_same<T, float>::value ? 1 : 4, threads = 1024 / ctas;
    const int grid = (int)std::min<long long>(M, (long long)ctas * std::max(1, p->sm_count));
    const size_t bytes = sizeof(V) * (size_t)stride * grid;
    if (p->adj_ws_bytes < bytes) {
        cudaFree(p->d_adj_ws);
        p->d_adj_ws = nullptr;
        p->adj_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&p->d_adj_ws, bytes);
        if (e != cudaSuccess) return set_cuda_error(e);
        p->adj_ws_bytes = bytes;
    }
    // the kernel accumulates with atomics: start from zero
    if (gU) zero_kernel<<<1, 32, 0, s>>>(gU, 1);
    if (gt && p->B) zero_kernel<<<(p->B + 255) / 256, 256, 0, s>>>(gt, p->B);
    if (gn) zero_kernel<<<(2 * N + 255) / 256, 256, 0, s>>>(gn, 2 * N);
    AdjArgs<T> a;
    a.N = N;
    a.B = p->B;
    a.NE = NE;
    a.nbr = p->d_nbr;
    a.nbr_bond = p->d_nbr_bond;
    a.bonds = p->d_bonds;
    a.tnb = std::is_same<T, double>::value ? reinterpret_cast<const T *>(p->d_t64)
                                           : reinterpret_cast<const T *>(p->d_t32);
    a.nocc = p->d_n;
    a.U = (T)p->U;
    a.dt = (T)p->dt;
    a.out_every = p->out_every;
    a.ckpt_every = ckpt_every;
    a.n_steps = n_steps;
    a.M = M;
    a.seed = seed;
    a.dL = dL;
    a.dS = dS;
    a.mu = mu;
    a.gU = gU;
    a.gt = gt;
    a.gn = gn;
    a.ws = reinterpret_cast<V *>(p->d_adj_ws);
    a.ws_stride = stride;
    a.status = p->d_status;
    const int smem = smem_tables;
    if (smem > 227 * 1024) return FTWA_ERR_UNSUPPORTED;
    auto kern = ctas == 4 ? adjoint_kernel<T, 256, 4> : adjoint_kernel<T, 1024, 1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return set_cuda_error(e);
    kern<<<grid, threads, smem, s>>>(a);
    return set_cuda_error(cudaGetLastError());
}

int launch_adjoint(Plan *p, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every, const double *dL,
                   const double *dC, const double *occ, double *gU, double *gt, double *gn, cudaStream_t s)
{
    // the samples of a general initial state depend on the eigenbasis, whose
    // derivatives the adjoint does not carry
    if (p->general_basis) return FTWA_ERR_UNSUPPORTED;
    // nor through the time-dependent drive or a long-range interaction
    if (p->drive || p->longrange || p->hop_drive) return FTWA_ERR_UNSUPPORTED;
    const double *dS = nullptr, *mu = nullptr;
    if (dC) {
        // S = G + G^T and mu = <n> - 1/2 for every output row, in the plan's
        // correlation workspace (grown on demand)
        const int K = 2 * p->N, T = (int)(n_steps / p->out_every) + 1;
        const size_t bytes = sizeof(double) * ((size_t)T * K * K + (size_t)T * K);
        if (p->corr_ws_bytes < bytes) {
            cudaFree(p->d_corr_ws);
            p->d_corr_ws = nullptr;
            p->corr_ws_bytes = 0;
            cudaError_t e = cudaMalloc(&p->d_corr_ws, bytes);
            if (e != cudaSuccess) return set_cuda_error(e);
            p->corr_ws_bytes = bytes;
        }
        double *S = static_cast<double *>(p->d_corr_ws);
        double *m = S + (size_t)T * K * K;
        const long long n = (long long)T * K * K;
        adj::symmetrise_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 8192), 256, 0, s>>>(dC, occ, T, K, S, m);
        const int rc = set_cuda_error(cudaGetLastError());
        if (rc != FTWA_OK) return rc;
        dS = S;
        mu = m;
    }
    if (p->precision == FTWA_FP64)
        return launch_adjoint_t<double>(p, seed, M, n_steps, ckpt_every, dL, dS, mu, gU, gt, gn, s);
    return launch_adjoint_t<float>(p, seed, M, n_steps, ckpt_every, dL, dS, mu, gU, gt, gn, s);
}

}  // namespace ftwa
