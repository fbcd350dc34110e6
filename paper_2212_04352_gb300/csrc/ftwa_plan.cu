// C ABI entry points: plan creation and validation, dispatch, status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "ftwa_internal.h"

namespace ftwa {

int set_cuda_error(cudaError_t e)
{
    if (e == cudaSuccess) return FTWA_OK;
    if (e == cudaErrorMemoryAllocation) return FTWA_ERR_OUT_OF_MEMORY;
    return FTWA_ERR_CUDA;
}

void free_drive(Plan *p)
{
    cudaFree(p->d_amp64);
    cudaFree(p->d_amp32);
    cudaFree(p->d_ftab);
    p->d_amp64 = nullptr;
    p->d_amp32 = nullptr;
    p->d_ftab = nullptr;
    p->ftab_bytes = 0;
    p->drive = false;
}

void free_interaction(Plan *p)
{
    cudaFree(p->d_u64);
    cudaFree(p->d_u32);
    p->d_u64 = nullptr;
    p->d_u32 = nullptr;
    p->longrange = false;
}

static void free_tables(Plan *p)
{
    cudaFree(p->d_nbr);
    cudaFree(p->d_nbr_bond);
    cudaFree(p->d_t64);
    cudaFree(p->d_t32);
    cudaFree(p->d_n);
    cudaFree(p->d_bonds);
    cudaFree(p->d_status);
    cudaFree(p->d_ws);
    cudaFree(p->d_items);
    cudaFree(p->d_tile);
    p->d_tile = nullptr;
    p->tile_bytes = 0;
    p->tile_host.clear();
    cudaFree(p->d_adj_ws);
    cudaFree(p->d_corr_ws);
    p->d_corr_ws = nullptr;
    p->corr_ws_bytes = 0;
    free_basis(p);
    free_drive(p);
    free_interaction(p);
    p->d_adj_ws = nullptr;
    p->adj_ws_bytes = 0;
    p->d_items = nullptr;
    p->items_bytes = 0;
    p->d_ws = nullptr;
    p->ws_bytes = 0;
    p->d_nbr = nullptr;
    p->d_nbr_bond = nullptr;
    p->d_t64 = nullptr;
    p->d_t32 = nullptr;
    p->d_n = nullptr;
    p->d_bonds = nullptr;
    p->d_status = nullptr;
}

template <typename X>
static int upload(X **dst, const X *src, size_t n)
{
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), std::max<size_t>(n, 1) * sizeof(X));
    if (e != cudaSuccess) return set_cuda_error(e);
    if (n) e = cudaMemcpy(*dst, src, n * sizeof(X), cudaMemcpyHostToDevice);
    return set_cuda_error(e);
}

// Two-colouring of the bond graph; false if it is not bipartite.
static bool two_colour(int N, const std::vector<int32_t> &bonds, std::vector<int> &col)
{
    std::vector<std::vector<int>> adj(N);
    for (size_t b = 0; b < bonds.size() / 2; ++b) {
        adj[bonds[2 * b]].push_back(bonds[2 * b + 1]);
        adj[bonds[2 * b + 1]].push_back(bonds[2 * b]);
    }
    col.assign(N, -1);
    for (int s0 = 0; s0 < N; ++s0) {
        if (col[s0] >= 0) continue;
        col[s0] = 0;
        std::vector<int> q{s0};
        for (size_t h = 0; h < q.size(); ++h) {
            for (int v : adj[q[h]]) {
                if (col[v] < 0) {
                    col[v] = 1 - col[q[h]];
                    q.push_back(v);
                } else if (col[v] == col[q[h]]) {
                    return false;
                }
            }
        }
    }
    return true;
}

// Slot order for shared-memory banks.  A warp of the banded stepper takes 32
// consecutive columns q = qoff + 32 blk + lane (qoff = N - 32 ceil(N/32);
// lanes with q < 0 take column 0) and, for each slot n, gathers
// rho_p,k(q,n) from one row p.  In FP32 (8-byte elements) a half-warp is
// served in one shared-memory wavefront when its distinct k are distinct
// mod 16; in FP64 (16-byte elements) a quarter-warp, mod 8.  The sum over a
// site's slots is order-free, so the real neighbours may be permuted among
// slots 0 .. deg-1 (the kernels take slots below the degree as bonds), and
// an empty slot (hopping 0) may point at any column within +-3 of the site
// and within the band (|k - i| <= bw, stored in every row that reads it).
// Greedy sweeps over these choices minimise, per group of columns, the
// wavefronts and then the sum of squared bank loads.
struct SlotSearch {
    int N, bw, qoff;
    const std::vector<int> &deg;
    std::vector<int> &slot_k;

    // first site and end (exclusive) of the column group of site i
    void group(int i, int w, int &g0, int &g1) const
    {
        const int g = (i - qoff) / w;
        g0 = std::max(0, qoff + g * w);
        g1 = std::min(N, qoff + (g + 1) * w);
    }
    double group_cost(int g0, int g1, int mod) const
    {
        double c = 0;
        for (int n = 0; n < 3; ++n) {
            int ks[16], nk = 0, cnt[16] = {0};
            for (int x = g0; x < g1; ++x) {
                const int k = slot_k[3 * x + n];
                bool seen = false;
                for (int y = 0; y < nk; ++y) seen = seen || ks[y] == k;
                if (!seen) {
                    ks[nk++] = k;
                    cnt[k % mod]++;
                }
            }
            int mx = 0, sq = 0;
            for (int b = 0; b < mod; ++b) {
                mx = std::max(mx, cnt[b]);
                sq += cnt[b] * cnt[b];
            }
            c += 64.0 * mx + sq;
        }
        return c;
    }
    double site_cost(int i) const
    {
        int a0, a1, b0, b1;
        group(i, 16, a0, a1);
        group(i, 8, b0, b1);
        return group_cost(a0, a1, 16) + 0.5 * group_cost(b0, b1, 8);
    }
};

static void order_slots_for_banks(int N, int bw, const std::vector<int> &deg, std::vector<int> &slot_k,
                                  std::vector<double> &t64, std::vector<int32_t> &bond)
{
    SlotSearch S{N, bw, N - 32 * ((N + 31) / 32), deg, slot_k};
    for (int sweep = 0; sweep < 8; ++sweep) {
        bool changed = false;
        for (int i = 0; i < N; ++i) {
            const int d = deg[i];
            int k0[3], b0[3];
            double t0[3];
            for (int n = 0; n < 3; ++n) {
                k0[n] = slot_k[3 * i + n];
                b0[n] = bond[3 * i + n];
                t0[n] = t64[4 * i + n];
            }
            std::vector<int> ph;   // placeholder columns
            for (int k = i - 3; k <= i + 3; ++k)
                if (k >= 0 && k < N && std::abs(k - i) <= bw) ph.push_back(k);
            double best = S.site_cost(i);
            int best_perm[3] = {0, 1, 2}, best_ph[3] = {k0[0], k0[1], k0[2]};
            int perm[3] = {0, 1, 2};
            do {
                int sel[3] = {0, 0, 0};   // odometer over the empty slots' columns
                while (true) {
                    for (int n = 0; n < 3; ++n) slot_k[3 * i + n] = n < d ? k0[perm[n]] : ph[sel[n]];
                    const double c = S.site_cost(i);
                    if (c < best - 1e-9) {
                        best = c;
                        for (int n = 0; n < 3; ++n) {
                            best_perm[n] = perm[n];
                            best_ph[n] = slot_k[3 * i + n];
                        }
                    }
                    int n = d;
                    while (n < 3 && ++sel[n] == (int)ph.size()) sel[n++] = 0;
                    if (n >= 3) break;
                }
            } while (std::next_permutation(perm, perm + d));
            for (int n = 0; n < 3; ++n) {
                if (n < d) {
                    slot_k[3 * i + n] = k0[best_perm[n]];
                    bond[3 * i + n] = b0[best_perm[n]];
                    t64[4 * i + n] = t0[best_perm[n]];
                } else {
                    slot_k[3 * i + n] = best_ph[n];
                }
                changed = changed || slot_k[3 * i + n] != k0[n];
            }
        }
        if (!changed) break;
    }
}

}  // namespace ftwa

using namespace ftwa;

extern "C" {

int ftwa_version(void) { return 10000; }

const char *ftwa_error_string(int status)
{
    switch (status) {
    case FTWA_OK: return "ok";
    case FTWA_ERR_INVALID_ARGUMENT: return "invalid argument";
    case FTWA_ERR_UNSUPPORTED: return "unsupported lattice or size";
    case FTWA_ERR_OUT_OF_MEMORY: return "device out of memory";
    case FTWA_ERR_CUDA: return "CUDA runtime error";
    case FTWA_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case FTWA_ERR_NONFINITE: return "non-finite value produced";
    default: return "unknown status";
    }
}

int ftwa_plan(const ftwa_lattice *lat, double U, double t, double filling, const ftwa_init_state *init,
              const ftwa_options *opts, ftwa_plan_t **out)
{
    if (!out || !lat) return FTWA_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    const int N = lat->n_sites, B = lat->n_bonds;
    if (N < 2 || N > FTWA_MAX_SITES) return FTWA_ERR_UNSUPPORTED;
    if (B < 0 || (B > 0 && !lat->bonds)) return FTWA_ERR_INVALID_ARGUMENT;
    if (!std::isfinite(U) || !std::isfinite(t)) return FTWA_ERR_INVALID_ARGUMENT;
    if (B > 3 * N) return FTWA_ERR_UNSUPPORTED;

    ftwa_options o{};
    if (opts) o = *opts;
    if (o.precision != FTWA_FP64 && o.precision != FTWA_FP32) return FTWA_ERR_INVALID_ARGUMENT;
    if (o.dt == 0.0) o.dt = 0.01;
    if (!(o.dt > 0.0) || !std::isfinite(o.dt)) return FTWA_ERR_INVALID_ARGUMENT;
    if (o.out_every == 0) o.out_every = 10;
    if (o.out_every < 1) return FTWA_ERR_INVALID_ARGUMENT;
    if (o.cluster_override < 0 || o.cluster_override > kMaxCluster ||
        (o.cluster_override & (o.cluster_override - 1)) != 0)
        return FTWA_ERR_INVALID_ARGUMENT;
    // 768 threads for every stepper; the tiled stepper also runs with 512
    if (o.threads_override != 0 && o.threads_override != kThreads && !(o.threads_override == 512 && o.variant == 3))
        return FTWA_ERR_UNSUPPORTED;
    if (o.variant < 0 || o.variant > 3) return FTWA_ERR_INVALID_ARGUMENT;

    ftwa_plan_t *p = new (std::nothrow) ftwa_plan_t();
    if (!p) return FTWA_ERR_OUT_OF_MEMORY;
    p->N = N;
    p->B = B;
    p->precision = o.precision;
    p->U = U;
    p->dt = o.dt;
    p->out_every = o.out_every;
    p->cluster_override = o.cluster_override;
    p->threads_override = o.threads_override;
    p->autotune = o.autotune;
    p->variant_override = o.variant;
    if (o.timeout_us) p->timeout_ns = o.timeout_us * 1000ull;

    // bonds: 0 <= i < j < N, unique, degree <= 3
    p->bonds.assign(lat->bonds, lat->bonds + 2 * (size_t)B);
    p->t_bond.resize(B);
    std::set<std::pair<int, int>> seen;
    std::vector<int> deg(N, 0);
    for (int b = 0; b < B; ++b) {
        const int i = p->bonds[2 * b], j = p->bonds[2 * b + 1];
        if (i < 0 || j >= N || i >= j || !seen.insert({i, j}).second) {
            delete p;
            return FTWA_ERR_INVALID_ARGUMENT;
        }
        const double tb = lat->t_bond ? lat->t_bond[b] : t;
        if (!std::isfinite(tb)) {
            delete p;
            return FTWA_ERR_INVALID_ARGUMENT;
        }
        p->t_bond[b] = tb;
        if (++deg[i] > 3 || ++deg[j] > 3) {
            delete p;
            return FTWA_ERR_UNSUPPORTED;
        }
    }
    p->bandwidth = 1;
    for (int b = 0; b < B; ++b) p->bandwidth = std::max(p->bandwidth, p->bonds[2 * b + 1] - p->bonds[2 * b]);
    p->uniform_t = true;
    for (int b = 1; b < B; ++b) p->uniform_t = p->uniform_t && p->t_bond[b] == p->t_bond[0];

    // occupations
    p->n_up.resize(N);
    p->n_dn.resize(N);
    if (init) {
        if (!init->n_up || !init->n_dn) {
            delete p;
            return FTWA_ERR_INVALID_ARGUMENT;
        }
        double tot = 0;
        for (int i = 0; i < N; ++i) {
            const double a = init->n_up[i], b = init->n_dn[i];
            if (!(a >= 0.0 && a <= 1.0 && b >= 0.0 && b <= 1.0)) {
                delete p;
                return FTWA_ERR_INVALID_ARGUMENT;
            }
            p->n_up[i] = a;
            p->n_dn[i] = b;
            tot += a + b;
        }
        if (filling > 0 && std::fabs(tot / (2.0 * N) - filling) > 1e-9) {
            delete p;
            return FTWA_ERR_INVALID_ARGUMENT;
        }
    } else {
        std::vector<int> col;
        if (filling != 0.5 || !two_colour(N, p->bonds, col)) {
            delete p;
            return FTWA_ERR_INVALID_ARGUMENT;
        }
        for (int i = 0; i < N; ++i) {
            p->n_up[i] = col[i] == col[0] ? 1.0 : 0.0;
            p->n_dn[i] = 1.0 - p->n_up[i];
        }
    }

    // neighbour tables: filled slots first; empty slots point at the site
    // itself with zero hopping
    p->nbr_host.assign(N, 0);
    p->nbr_bond.assign(3 * (size_t)N, -1);
    std::vector<double> t64(4 * (size_t)N, 0.0);
    std::vector<int> fill(N, 0);
    std::vector<int> slot_k(3 * (size_t)N);
    for (int i = 0; i < N; ++i)
        for (int n = 0; n < 3; ++n) slot_k[3 * i + n] = i;
    for (int b = 0; b < B; ++b) {
        const int i = p->bonds[2 * b], j = p->bonds[2 * b + 1];
        slot_k[3 * i + fill[i]] = j;
        t64[4 * i + fill[i]] = p->t_bond[b];
        p->nbr_bond[3 * i + fill[i]] = b;
        fill[i]++;
        slot_k[3 * j + fill[j]] = i;
        t64[4 * j + fill[j]] = p->t_bond[b];
        p->nbr_bond[3 * j + fill[j]] = b;
        fill[j]++;
    }
    // order each site's slots by distance |k - i| (then k): the starting point
    // of order_slots_for_banks (on lattices numbered along rows, slots 0 and 1
    // are then the in-row neighbours i -+ 1 for most sites)
    for (int i = 0; i < N; ++i) {
        int idx[3] = {0, 1, 2};
        std::sort(idx, idx + fill[i], [&](int x, int y) {
            const int kx = slot_k[3 * i + x], ky = slot_k[3 * i + y];
            const int dx = std::abs(kx - i), dy = std::abs(ky - i);
            return dx != dy ? dx < dy : kx < ky;
        });
        int k2[3], b2[3];
        double t2[3];
        for (int n = 0; n < 3; ++n) {
            const int src = n < fill[i] ? idx[n] : n;
            k2[n] = slot_k[3 * i + src];
            b2[n] = p->nbr_bond[3 * i + src];
            t2[n] = t64[4 * i + src];
        }
        for (int n = 0; n < 3; ++n) {
            slot_k[3 * i + n] = k2[n];
            p->nbr_bond[3 * i + n] = b2[n];
            t64[4 * i + n] = t2[n];
        }
    }
    order_slots_for_banks(N, p->bandwidth, fill, slot_k, t64, p->nbr_bond);
    for (int i = 0; i < N; ++i)
        p->nbr_host[i] = slot_k[3 * i] | (slot_k[3 * i + 1] << 8) | (slot_k[3 * i + 2] << 16) | (fill[i] << 24);
    std::vector<float> t32(t64.begin(), t64.end());
    std::vector<double> nn(2 * (size_t)N);
    for (int i = 0; i < N; ++i) {
        nn[i] = p->n_up[i];
        nn[N + i] = p->n_dn[i];
    }

    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return set_cuda_error(e);
    }
    int rc = upload(&p->d_nbr, p->nbr_host.data(), N);
    if (rc == FTWA_OK) rc = upload(&p->d_nbr_bond, p->nbr_bond.data(), 3 * (size_t)N);
    if (rc == FTWA_OK) rc = upload(&p->d_t64, t64.data(), t64.size());
    if (rc == FTWA_OK) rc = upload(&p->d_t32, t32.data(), t32.size());
    if (rc == FTWA_OK) rc = upload(&p->d_n, nn.data(), nn.size());
    if (rc == FTWA_OK) rc = upload(&p->d_bonds, p->bonds.data(), p->bonds.size());
    if (rc == FTWA_OK) {
        e = cudaMalloc(&p->d_status, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
        rc = set_cuda_error(e);
    }
    if (rc != FTWA_OK) {
        free_tables(p);
        delete p;
        return rc;
    }
    {
        BandShape bs;
        const bool try_band = p->variant_override == 1 || (p->variant_override == 0 && p->precision == FTWA_FP32);
        if (p->variant_override == 3 || (p->variant_override == 0 && tile_supported(p))) {
            // shape of the tiled stepper for one sample per cluster (tables are
            // built and uploaded by the first evolve)
            p->dry_run = true;
            rc = launch_tile(p, nullptr, (int64_t)p->sm_count, 1, nullptr, nullptr);
            p->dry_run = false;
            if (rc == FTWA_OK || p->variant_override == 3) goto shape_done;
        }
        if (try_band && choose_band_shape(p, (int64_t)p->sm_count, &bs) == FTWA_OK) {
            p->shape.cluster = bs.cluster;
            p->shape.slots = bs.slots;
            p->shape.units_per_warp = bs.E;
            p->shape.smem_bytes = bs.smem_bytes;
            p->shape.grid = bs.grid;
            p->shape.variant = 1;
            p->shape.threads = kThreads;
            rc = FTWA_OK;
        } else if (p->variant_override == 1) {
            rc = FTWA_ERR_UNSUPPORTED;
        } else {
            rc = choose_stepper_shape(p, (int64_t)p->sm_count, &p->shape);
            p->shape.variant = 2;
        }
    }
shape_done:
    if (rc != FTWA_OK) {
        free_tables(p);
        delete p;
        return rc;
    }
    *out = p;
    return FTWA_OK;
}

void ftwa_destroy(ftwa_plan_t *p)
{
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    free_tables(p);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
}

int ftwa_get_info(const ftwa_plan_t *p, ftwa_plan_info *info)
{
    if (!p || !info) return FTWA_ERR_INVALID_ARGUMENT;
    info->n_sites = p->N;
    info->n_bonds = p->B;
    info->precision = p->precision;
    info->cluster = p->shape.cluster;
    info->threads = p->shape.threads;
    info->samples_per_cta = p->shape.slots;
    info->smem_bytes = p->shape.smem_bytes;
    info->tmem_cols = kTmemCols;
    info->grid_clusters = p->shape.grid / std::max(1, p->shape.cluster);
    info->units_per_warp = p->shape.units_per_warp;
    info->variant = p->shape.variant;
    return FTWA_OK;
}

int ftwa_sample(ftwa_plan_t *p, uint64_t seed, int64_t first_sample, int64_t M, void *rho_dev, void *stream)
{
    if (!p || M < 0 || first_sample < 0 || (M > 0 && !rho_dev)) return FTWA_ERR_INVALID_ARGUMENT;
    return launch_sample(p, seed, first_sample, M, rho_dev, static_cast<cudaStream_t>(stream));
}

int ftwa_philox(uint64_t seed, int64_t m, int32_t spin, int64_t p0, int64_t count, uint32_t *out_dev, void *stream)
{
    if (count < 0 || m < 0 || p0 < 0 || (count > 0 && !out_dev)) return FTWA_ERR_INVALID_ARGUMENT;
    return launch_philox(seed, m, spin, p0, count, out_dev, static_cast<cudaStream_t>(stream));
}

int ftwa_evolve(ftwa_plan_t *p, void *rho_dev, int64_t M, int64_t n_steps, void *snap_dev, void *stream)
{
    if (!p || M < 0 || n_steps < 0 || (M > 0 && !rho_dev)) return FTWA_ERR_INVALID_ARGUMENT;
    return launch_evolve(p, rho_dev, M, n_steps, snap_dev, static_cast<cudaStream_t>(stream));
}

int ftwa_evolve_at(ftwa_plan_t *p, void *rho_dev, int64_t M, int64_t n_steps, double t_start, void *snap_dev,
                   void *stream)
{
    if (!p || M < 0 || n_steps < 0 || (M > 0 && !rho_dev) || !std::isfinite(t_start))
        return FTWA_ERR_INVALID_ARGUMENT;
    return launch_evolve(p, rho_dev, M, n_steps, snap_dev, static_cast<cudaStream_t>(stream), t_start);
}

int ftwa_set_hopping_drive(ftwa_plan_t *p, double eps, double t0, double sigma, double omega, double phase)
{
    if (!p || !std::isfinite(eps) || !std::isfinite(t0) || !std::isfinite(sigma) || !std::isfinite(omega) ||
        !std::isfinite(phase))
        return FTWA_ERR_INVALID_ARGUMENT;
    p->hop_drive = eps != 0.0;
    p->hop_eps = eps;
    p->hop_t0 = t0;
    p->hop_sigma = sigma;
    p->hop_omega = omega;
    p->hop_phase = phase;
    return FTWA_OK;
}

int ftwa_set_interaction(ftwa_plan_t *p, const double *u)
{
    if (!p) return FTWA_ERR_INVALID_ARGUMENT;
    if (!u) {
        free_interaction(p);
        return FTWA_OK;
    }
    const int N = p->N;
    double scale = 0.0;
    for (size_t k = 0; k < (size_t)N * N; ++k) {
        if (!std::isfinite(u[k])) return FTWA_ERR_INVALID_ARGUMENT;
        scale = std::max(scale, std::fabs(u[k]));
    }
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            if (std::fabs(u[(size_t)i * N + j] - u[(size_t)j * N + i]) > 1e-12 * std::max(scale, 1.0))
                return FTWA_ERR_INVALID_ARGUMENT;
    free_interaction(p);
    const size_t n = (size_t)N * N;
    std::vector<float> u32(u, u + n);
    cudaError_t e = cudaMalloc(&p->d_u64, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_u64, u, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_u32, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_u32, u32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_interaction(p);
        return set_cuda_error(e);
    }
    p->longrange = true;
    return FTWA_OK;
}

int ftwa_set_drive(ftwa_plan_t *p, const double *amp, double t0, double sigma, double omega, double phase)
{
    if (!p) return FTWA_ERR_INVALID_ARGUMENT;
    if (!amp) {
        free_drive(p);
        return FTWA_OK;
    }
    if (!std::isfinite(t0) || !std::isfinite(sigma) || !std::isfinite(omega) || !std::isfinite(phase))
        return FTWA_ERR_INVALID_ARGUMENT;
    const int n = 2 * p->N;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(amp[i])) return FTWA_ERR_INVALID_ARGUMENT;
    free_drive(p);
    std::vector<float> a32(amp, amp + n);
    cudaError_t e = cudaMalloc(&p->d_amp64, sizeof(double) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_amp64, amp, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_amp32, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_amp32, a32.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_drive(p);
        return set_cuda_error(e);
    }
    p->drive_t0 = t0;
    p->drive_sigma = sigma;
    p->drive_omega = omega;
    p->drive_phase = phase;
    p->drive = true;
    return FTWA_OK;
}

int ftwa_moments(ftwa_plan_t *p, const void *snap_dev, int64_t M, int32_t n_times, double *occ_dev, double *conn_dev,
                 double *g2_dev, int32_t gram_mode, void *stream)
{
    if (!p || !snap_dev || M < 1 || n_times < 1 || !occ_dev || !conn_dev) return FTWA_ERR_INVALID_ARGUMENT;
    if (gram_mode != FTWA_GRAM_FP64 && gram_mode != FTWA_GRAM_BF16X3) return FTWA_ERR_INVALID_ARGUMENT;
    return launch_moments(p, snap_dev, M, n_times, occ_dev, conn_dev, g2_dev, gram_mode,
                          static_cast<cudaStream_t>(stream));
}

int ftwa_adjoint(ftwa_plan_t *p, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every,
                 const double *dL_docc_dev, double *grad_U_dev, double *grad_t_dev, double *grad_n0_dev, void *stream)
{
    if (!p || M < 1 || n_steps < 1 || ckpt_every < 1 || !dL_docc_dev) return FTWA_ERR_INVALID_ARGUMENT;
    if (n_steps % ckpt_every != 0 || ckpt_every % p->out_every != 0) return FTWA_ERR_INVALID_ARGUMENT;
    return launch_adjoint(p, seed, M, n_steps, ckpt_every, dL_docc_dev, nullptr, nullptr, grad_U_dev, grad_t_dev,
                          grad_n0_dev, static_cast<cudaStream_t>(stream));
}

int ftwa_adjoint_corr(ftwa_plan_t *p, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every,
                      const double *dL_docc_dev, const double *dL_dconn_dev, const double *occ_dev,
                      double *grad_U_dev, double *grad_t_dev, double *grad_n0_dev, void *stream)
{
    if (!p || M < 1 || n_steps < 1 || ckpt_every < 1) return FTWA_ERR_INVALID_ARGUMENT;
    if (!dL_docc_dev && !dL_dconn_dev) return FTWA_ERR_INVALID_ARGUMENT;
    if (dL_dconn_dev && !occ_dev) return FTWA_ERR_INVALID_ARGUMENT;
    if (n_steps % ckpt_every != 0 || ckpt_every % p->out_every != 0) return FTWA_ERR_INVALID_ARGUMENT;
    return launch_adjoint(p, seed, M, n_steps, ckpt_every, dL_docc_dev, dL_dconn_dev, occ_dev, grad_U_dev,
                          grad_t_dev, grad_n0_dev, static_cast<cudaStream_t>(stream));
}

int ftwa_status(ftwa_plan_t *p, void *stream)
{
    if (!p) return FTWA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return FTWA_ERR_CUDA;
    int v = 0;
    e = cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return FTWA_ERR_CUDA;
    return v;
}

int ftwa_debug_force_timeout(ftwa_plan_t *p, int32_t armed)
{
    if (!p) return FTWA_ERR_INVALID_ARGUMENT;
    p->force_timeout = armed ? 1 : 0;
    return FTWA_OK;
}

}  // extern "C"
