// Exact diagonalisation reference on the GPU (Sec. III.A and App. B: the
// comparison method of the paper, for 10-16-site lattices).
//
// The many-body state of Eq. 1 with fixed N_up, N_dn is a dim_up x dim_dn
// complex matrix psi[a][b] over Slater determinants (a: spin-up
// configuration, b: spin-down configuration, configurations as bit masks in
// increasing order).  H psi = T_up psi + psi T_dn^T + U D o psi with the
// single-species hopping matrices T_s (CSR, built on the host when the plan
// is made: -t_b times the fermionic sign (-1)^(occupied same-spin orbitals
// strictly between the two sites)) and D[a][b] = popcount(a & b).  Time
// evolution psi(t) = exp(-iHt) psi(0) (the Schroedinger form) by a
// Chebyshev expansion over intervals dt_out: with H~ = (H - b)/a (spectrum
// in [-1, 1]), exp(-iH dt) = exp(-ib dt) sum_k (2 - delta_k0) (-i)^k
// J_k(a dt) T_k(H~).  The recurrence T_{k+1} = 2 H~ T_k - T_{k-1} and the
// accumulation of the sum are fused into one kernel per term.  Observables
// per output time: <n_i,s> and <n_a n_b> over the 2N site-spins.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ftwa_internal.h"

namespace ftwa {
namespace ed {

constexpr int kMaxSitesEd = 24;   // configurations are 32-bit masks; dims grow as C(N, N/2)^2

// plain view of the plan, passed to the kernels by value
struct EdView {
    int N;
    long long dim_up, dim_dn, dim;
    double U, a, b;                           // spectral map H~ = (H - b) / a
    const uint32_t *conf_up, *conf_dn;        // configuration bit masks
    const int *rp_up, *ci_up, *rp_dn, *ci_dn; // CSR of T_up, T_dn
    const double *v_up, *v_dn;
    double *pu, *pd;                          // marginals of |psi|^2 over the other species
    double *q;                                // [dim_up][N]: sum_b |psi_ab|^2 n_j(b)
};

}  // namespace ed
}  // namespace ftwa

struct ftwa_ed {
    int N = 0, n_up = 0, n_dn = 0;
    std::vector<uint32_t> conf_up, conf_dn;
    ftwa::ed::EdView v{};
    uint32_t *d_conf_up = nullptr, *d_conf_dn = nullptr;
    int *d_rp_up = nullptr, *d_ci_up = nullptr, *d_rp_dn = nullptr, *d_ci_dn = nullptr;
    double *d_v_up = nullptr, *d_v_dn = nullptr;
    double2 *d_psi = nullptr, *d_t0 = nullptr, *d_t1 = nullptr, *d_t2 = nullptr;
    double *d_pu = nullptr, *d_pd = nullptr, *d_q = nullptr;
};

namespace ftwa {
namespace ed {

// hop T: y[a][b] gets sum over the row of T_up (a) of v * x[a'][b] and over
// the row of T_dn (b) of v * x[a][b']; plus U popc(a & b) x[a][b]
__device__ __forceinline__ double2 apply_h(const EdView &e, const double2 *__restrict__ x, long long ia, long long ib)
{
    double2 y = make_double2(0.0, 0.0);
    for (int k = e.rp_up[ia]; k < e.rp_up[ia + 1]; ++k) {
        const double2 v = x[(long long)e.ci_up[k] * e.dim_dn + ib];
        y.x = fma(e.v_up[k], v.x, y.x);
        y.y = fma(e.v_up[k], v.y, y.y);
    }
    for (int k = e.rp_dn[ib]; k < e.rp_dn[ib + 1]; ++k) {
        const double2 v = x[ia * e.dim_dn + e.ci_dn[k]];
        y.x = fma(e.v_dn[k], v.x, y.x);
        y.y = fma(e.v_dn[k], v.y, y.y);
    }
    const double d = e.U * (double)__popc(e.conf_up[ia] & e.conf_dn[ib]);
    const double2 v = x[ia * e.dim_dn + ib];
    y.x = fma(d, v.x, y.x);
    y.y = fma(d, v.y, y.y);
    return y;
}

// Chebyshev term: tn = first ? H~ tc : 2 H~ tc - tp; acc += c tn (c complex)
__global__ void cheb_kernel(EdView e, const double2 *__restrict__ tc, const double2 *__restrict__ tp,
                            double2 *__restrict__ tn, double2 *__restrict__ acc, double cr, double ci, int first)
{
    const long long total = e.dim;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long ia = i / e.dim_dn, ib = i % e.dim_dn;
        const double2 h = apply_h(e, tc, ia, ib);
        const double2 c = tc[i];
        double2 w;
        w.x = (h.x - e.b * c.x) / e.a;
        w.y = (h.y - e.b * c.y) / e.a;
        if (!first) {
            w.x = 2.0 * w.x - tp[i].x;
            w.y = 2.0 * w.y - tp[i].y;
        }
        tn[i] = w;
        double2 r = acc[i];
        r.x += cr * w.x - ci * w.y;
        r.y += cr * w.y + ci * w.x;
        acc[i] = r;
    }
}

// acc = c0 * t0 (the k = 0 term), t0 = psi
__global__ void cheb_init_kernel(long long n, const double2 *__restrict__ psi, double2 *__restrict__ t0,
                                 double2 *__restrict__ acc, double cr, double ci)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = psi[i];
        t0[i] = v;
        acc[i] = make_double2(cr * v.x - ci * v.y, cr * v.y + ci * v.x);
    }
}

// marginals: pu[a] = sum_b |psi|^2, q[a][j] = sum_b |psi|^2 n_j(b) (block per a)
__global__ void marg_up_kernel(EdView e, const double2 *__restrict__ psi)
{
    __shared__ double red[32][kMaxSitesEd + 1];
    const long long ia = blockIdx.x;
    const int N = e.N;
    double p = 0.0, q[kMaxSitesEd];
#pragma unroll
    for (int j = 0; j < kMaxSitesEd; ++j) q[j] = 0.0;
    for (long long ib = threadIdx.x; ib < e.dim_dn; ib += blockDim.x) {
        const double2 v = psi[ia * e.dim_dn + ib];
        const double w = v.x * v.x + v.y * v.y;
        p += w;
        const uint32_t cb = e.conf_dn[ib];
#pragma unroll
        for (int j = 0; j < kMaxSitesEd; ++j)
            if ((cb >> j) & 1u) q[j] += w;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
#pragma unroll
    for (int j = 0; j < kMaxSitesEd; ++j)
        for (int o = 16; o > 0; o >>= 1) q[j] += __shfl_xor_sync(0xffffffffu, q[j], o);
    if (lane == 0) {
        red[warp][kMaxSitesEd] = p;
#pragma unroll
        for (int j = 0; j < kMaxSitesEd; ++j) red[warp][j] = q[j];
    }
    __syncthreads();
    if (threadIdx.x <= kMaxSitesEd) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        if (threadIdx.x == kMaxSitesEd) e.pu[ia] = s;
        else if ((int)threadIdx.x < N) e.q[ia * N + threadIdx.x] = s;
    }
}

__global__ void marg_dn_kernel(EdView e, const double2 *__restrict__ psi)
{
    for (long long ib = blockIdx.x * (long long)blockDim.x + threadIdx.x; ib < e.dim_dn;
         ib += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long ia = 0; ia < e.dim_up; ++ia) {
            const double2 v = psi[ia * e.dim_dn + ib];
            s += v.x * v.x + v.y * v.y;
        }
        e.pd[ib] = s;
    }
}

// observables of one output time from the marginals (one block, 2N x 2N)
__global__ void observe_kernel(EdView e, double *occ, double *nn)
{
    const int N = e.N, K = 2 * N;
    for (int idx = threadIdx.x; idx < K * K + K; idx += blockDim.x) {
        double s = 0.0;
        if (idx >= K * K) {          // occupations
            const int k = idx - K * K;
            if (k < N) {
                for (long long ia = 0; ia < e.dim_up; ++ia)
                    if ((e.conf_up[ia] >> k) & 1u) s += e.pu[ia];
            } else {
                for (long long ib = 0; ib < e.dim_dn; ++ib)
                    if ((e.conf_dn[ib] >> (k - N)) & 1u) s += e.pd[ib];
            }
            occ[k] = s;
            continue;
        }
        if (!nn) continue;
        const int r = idx / K, c = idx % K;
        if (r < N && c < N) {                       // up-up
            for (long long ia = 0; ia < e.dim_up; ++ia) {
                const uint32_t ca = e.conf_up[ia];
                if (((ca >> r) & 1u) && ((ca >> c) & 1u)) s += e.pu[ia];
            }
        } else if (r >= N && c >= N) {              // dn-dn
            for (long long ib = 0; ib < e.dim_dn; ++ib) {
                const uint32_t cb = e.conf_dn[ib];
                if (((cb >> (r - N)) & 1u) && ((cb >> (c - N)) & 1u)) s += e.pd[ib];
            }
        } else {                                    // up-dn
            const int iu = r < N ? r : c, jd = r < N ? c - N : r - N;
            for (long long ia = 0; ia < e.dim_up; ++ia)
                if ((e.conf_up[ia] >> iu) & 1u) s += e.q[ia * N + jd];
        }
        nn[idx] = s;
    }
}

}  // namespace ed
}  // namespace ftwa

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

using namespace ftwa;

std::vector<uint32_t> configurations(int N, int n)
{
    std::vector<uint32_t> out;
    if (n == 0) {
        out.push_back(0u);
        return out;
    }
    uint32_t c = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    const uint64_t limit = 1ull << N;
    while ((uint64_t)c < limit) {
        out.push_back(c);
        const uint32_t t = c | (c - 1u);   // next mask with the same popcount (Gosper)
        const uint64_t nxt = (uint64_t)(t + 1u) | (((uint64_t)(~t & (t + 1u)) - 1u) >> (__builtin_ctz(c) + 1));
        if (t == 0xFFFFFFFFu || nxt >= limit) break;
        c = (uint32_t)nxt;
    }
    return out;
}

// CSR of the single-species hopping T = -sum_b t_b (c+_i c_j + c+_j c_i)
// over the configurations (symmetric: row c holds every c' reached from c);
// returns the largest absolute row sum (a bound of ||T||)
double hopping_csr(int N, const std::vector<uint32_t> &conf, const std::vector<int32_t> &bonds,
                   const std::vector<double> &tb, std::vector<int> &rp, std::vector<int> &ci, std::vector<double> &v)
{
    rp.assign(conf.size() + 1, 0);
    ci.clear();
    v.clear();
    double rmax = 0.0;
    for (size_t r = 0; r < conf.size(); ++r) {
        const uint32_t c = conf[r];
        double rs = 0.0;
        for (size_t b = 0; b < tb.size(); ++b) {
            for (int o = 0; o < 2; ++o) {
                const int i = o ? bonds[2 * b + 1] : bonds[2 * b], j = o ? bonds[2 * b] : bonds[2 * b + 1];
                if (!((c >> j) & 1u) || ((c >> i) & 1u)) continue;   // c+_i c_j needs j filled, i empty
                const int lo = std::min(i, j), hi = std::max(i, j);
                const uint32_t between = (hi - lo > 1) ? (((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u)) : 0u;
                const double sign = (__builtin_popcount(c & between) & 1) ? -1.0 : 1.0;
                const uint32_t c2 = (c & ~(1u << j)) | (1u << i);
                const size_t col = std::lower_bound(conf.begin(), conf.end(), c2) - conf.begin();
                ci.push_back((int)col);
                v.push_back(-tb[b] * sign);
                rs += std::fabs(tb[b]);
            }
        }
        rp[r + 1] = (int)ci.size();
        rmax = std::max(rmax, rs);
    }
    return rmax;
}

template <typename X>
int upload_vec(X **dst, const std::vector<X> &src)
{
    cudaError_t e = cudaMalloc(dst, sizeof(X) * std::max<size_t>(src.size(), 1));
    if (e == cudaSuccess && !src.empty()) e = cudaMemcpy(*dst, src.data(), sizeof(X) * src.size(), cudaMemcpyHostToDevice);
    return set_cuda_error(e);
}

void free_ed(ftwa_ed *p)
{
    cudaFree(p->d_conf_up);
    cudaFree(p->d_conf_dn);
    cudaFree(p->d_rp_up);
    cudaFree(p->d_ci_up);
    cudaFree(p->d_rp_dn);
    cudaFree(p->d_ci_dn);
    cudaFree(p->d_v_up);
    cudaFree(p->d_v_dn);
    cudaFree(p->d_psi);
    cudaFree(p->d_t0);
    cudaFree(p->d_t1);
    cudaFree(p->d_t2);
    cudaFree(p->d_pu);
    cudaFree(p->d_pd);
    cudaFree(p->d_q);
    delete p;
}

int grid_of(long long n)
{
    const long long g = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 16));
}

}  // namespace

extern "C" {

int ftwa_ed_plan(const ftwa_lattice *lat, double U, int32_t n_up, int32_t n_dn, ftwa_ed_t **out)
{
    if (!out || !lat || !lat->bonds || lat->n_sites < 1 || lat->n_bonds < 0) return FTWA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    const int N = lat->n_sites;
    if (N > ed::kMaxSitesEd) return FTWA_ERR_UNSUPPORTED;
    if (n_up < 0 || n_dn < 0 || n_up > N || n_dn > N || !std::isfinite(U)) return FTWA_ERR_INVALID_ARGUMENT;
    std::vector<int32_t> bonds(lat->bonds, lat->bonds + 2 * (size_t)lat->n_bonds);
    std::vector<double> tb(lat->n_bonds, 1.0);
    for (int b = 0; b < lat->n_bonds; ++b) {
        if (lat->t_bond) tb[b] = lat->t_bond[b];
        const int i = bonds[2 * b], j = bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j || !std::isfinite(tb[b])) return FTWA_ERR_INVALID_ARGUMENT;
    }
    ftwa_ed *p = new (std::nothrow) ftwa_ed;
    if (!p) return FTWA_ERR_OUT_OF_MEMORY;
    p->N = N;
    p->n_up = n_up;
    p->n_dn = n_dn;
    p->conf_up = configurations(N, n_up);
    p->conf_dn = configurations(N, n_dn);
    std::vector<int> rpu, ciu, rpd, cid;
    std::vector<double> vu, vd;
    const double ru = hopping_csr(N, p->conf_up, bonds, tb, rpu, ciu, vu);
    const double rd = hopping_csr(N, p->conf_dn, bonds, tb, rpd, cid, vd);
    ed::EdView &v = p->v;
    v.N = N;
    v.dim_up = (long long)p->conf_up.size();
    v.dim_dn = (long long)p->conf_dn.size();
    v.dim = v.dim_up * v.dim_dn;
    v.U = U;
    const double um = U * (double)std::min(n_up, n_dn);
    const double emax = ru + rd + std::max(0.0, um), emin = -ru - rd + std::min(0.0, um);
    v.b = 0.5 * (emax + emin);
    v.a = 0.5 * (emax - emin) * 1.01 + 1e-9;
    int rc = upload_vec(&p->d_conf_up, p->conf_up);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_conf_dn, p->conf_dn);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_rp_up, rpu);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_ci_up, ciu);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_v_up, vu);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_rp_dn, rpd);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_ci_dn, cid);
    if (rc == FTWA_OK) rc = upload_vec(&p->d_v_dn, vd);
    cudaError_t e = cudaSuccess;
    const size_t vb = sizeof(double2) * (size_t)v.dim;
    if (rc == FTWA_OK) {
        e = cudaMalloc(&p->d_psi, vb);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_t0, vb);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_t1, vb);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_t2, vb);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_pu, sizeof(double) * (size_t)v.dim_up);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_pd, sizeof(double) * (size_t)v.dim_dn);
        if (e == cudaSuccess) e = cudaMalloc(&p->d_q, sizeof(double) * (size_t)v.dim_up * N);
        rc = set_cuda_error(e);
    }
    if (rc != FTWA_OK) {
        free_ed(p);
        return rc;
    }
    v.conf_up = p->d_conf_up;
    v.conf_dn = p->d_conf_dn;
    v.rp_up = p->d_rp_up;
    v.ci_up = p->d_ci_up;
    v.v_up = p->d_v_up;
    v.rp_dn = p->d_rp_dn;
    v.ci_dn = p->d_ci_dn;
    v.v_dn = p->d_v_dn;
    v.pu = p->d_pu;
    v.pd = p->d_pd;
    v.q = p->d_q;
    *out = p;
    return FTWA_OK;
}

void ftwa_ed_destroy(ftwa_ed_t *p)
{
    if (p) {
        cudaDeviceSynchronize();
        free_ed(p);
    }
}

int ftwa_ed_info(const ftwa_ed_t *p, int64_t *dim, double *spectral_a, double *spectral_b)
{
    if (!p || !dim) return FTWA_ERR_INVALID_ARGUMENT;
    *dim = p->v.dim;
    if (spectral_a) *spectral_a = p->v.a;
    if (spectral_b) *spectral_b = p->v.b;
    return FTWA_OK;
}

int ftwa_ed_evolve(ftwa_ed_t *p, const double *n_up, const double *n_dn, double dt_out, int32_t n_out, double *occ_dev,
                   double *nn_dev, void *stream)
{
    if (!p || !n_up || !n_dn || !occ_dev || n_out < 0 || !(dt_out > 0.0) || !std::isfinite(dt_out))
        return FTWA_ERR_INVALID_ARGUMENT;
    const int N = p->N;
    uint32_t mu = 0, md = 0;
    for (int i = 0; i < N; ++i) {
        if (n_up[i] != 0.0 && n_up[i] != 1.0) return FTWA_ERR_INVALID_ARGUMENT;
        if (n_dn[i] != 0.0 && n_dn[i] != 1.0) return FTWA_ERR_INVALID_ARGUMENT;
        if (n_up[i] == 1.0) mu |= 1u << i;
        if (n_dn[i] == 1.0) md |= 1u << i;
    }
    if (__builtin_popcount(mu) != p->n_up || __builtin_popcount(md) != p->n_dn) return FTWA_ERR_INVALID_ARGUMENT;
    const long long ia = std::lower_bound(p->conf_up.begin(), p->conf_up.end(), mu) - p->conf_up.begin();
    const long long ib = std::lower_bound(p->conf_dn.begin(), p->conf_dn.end(), md) - p->conf_dn.begin();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const ed::EdView &v = p->v;
    const size_t vb = sizeof(double2) * (size_t)v.dim;
    cudaError_t e = cudaMemsetAsync(p->d_psi, 0, vb, s);
    const double2 one = make_double2(1.0, 0.0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_psi + ia * v.dim_dn + ib, &one, sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return set_cuda_error(e);
    // Chebyshev coefficients of exp(-iH dt) (one interval; identical for all)
    const double x = v.a * dt_out;
    std::vector<double> cr, ci;
    const double ph_r = std::cos(v.b * dt_out), ph_i = -std::sin(v.b * dt_out);   // exp(-i b dt)
    for (int k = 0; k < 100000; ++k) {
        const double jk = std::cyl_bessel_j((double)k, x);
        if (k > x + 10 && std::fabs(jk) < 1e-17) break;
        const double w = (k == 0 ? 1.0 : 2.0) * jk;
        // (-i)^k
        const int km = k & 3;
        const double pr = km == 0 ? 1.0 : (km == 2 ? -1.0 : 0.0), pi = km == 1 ? -1.0 : (km == 3 ? 1.0 : 0.0);
        cr.push_back(w * (pr * ph_r - pi * ph_i));
        ci.push_back(w * (pr * ph_i + pi * ph_r));
    }
    const int K = (int)cr.size();
    const int g = grid_of(v.dim);
    auto observe = [&](int row) -> int {
        ed::marg_up_kernel<<<(unsigned)v.dim_up, 256, 0, s>>>(v, p->d_psi);
        ed::marg_dn_kernel<<<grid_of(v.dim_dn), 256, 0, s>>>(v, p->d_psi);
        const int K2 = 2 * N;
        ed::observe_kernel<<<1, 256, 0, s>>>(v, occ_dev + (size_t)row * K2,
                                            nn_dev ? nn_dev + (size_t)row * K2 * K2 : nullptr);
        return set_cuda_error(cudaGetLastError());
    };
    int rc = observe(0);
    for (int t = 1; t <= n_out && rc == FTWA_OK; ++t) {
        double2 *acc = p->d_t0, *tp = p->d_psi, *tc = p->d_t1, *tn = p->d_t2;
        ed::cheb_init_kernel<<<g, 256, 0, s>>>(v.dim, p->d_psi, tp, acc, cr[0], ci[0]);
        // note: tp aliases psi (cheb_init copies psi onto itself); T_1 = H~ psi
        if (K > 1) ed::cheb_kernel<<<g, 256, 0, s>>>(v, tp, nullptr, tc, acc, cr[1], ci[1], 1);
        for (int k = 2; k < K; ++k) {
            ed::cheb_kernel<<<g, 256, 0, s>>>(v, tc, tp, tn, acc, cr[k], ci[k], 0);
            double2 *tmp = tp;
            tp = tc;
            tc = tn;
            tn = tmp;
        }
        rc = set_cuda_error(cudaGetLastError());
        // psi <- acc (the buffers rotate; psi keeps its role)
        std::swap(p->d_psi, p->d_t0);
        if (rc == FTWA_OK) rc = observe(t);
    }
    return rc;
}

}  // extern "C"
