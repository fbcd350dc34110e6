// Gaussian Wigner samples of a diagonal state (Eq. 7) from a counter-based
// generator.  Philox4x32-10 follows its published definition (Salmon,
// Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplies with
// the multipliers 0xD2511F53 / 0xCD9E8D57, the key bumped by the Weyl
// constants 0x9E3779B9 / 0xBB67AE85 between rounds.
#include <cuda_runtime.h>

#include "ftwa_internal.h"

namespace ftwa {

struct Philox4 {
    uint32_t x[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1)
{
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
    Philox4 o;
    o.x[0] = c0;
    o.x[1] = c1;
    o.x[2] = c2;
    o.x[3] = c3;
    return o;
}

// xi * sd for the pair index p of sample m, spin s.  u1, u2 are 53-bit
// uniforms in (0, 1); Box-Muller gives a, b ~ N(0, 1) and xi = (a + i b)/sqrt(2).
__device__ __forceinline__ double2 pair_value(uint64_t seed, long long m, int s, uint32_t p, double sd, double)
{
    const Philox4 w = philox4x32_10((uint32_t)m, (uint32_t)((unsigned long long)m >> 32), (uint32_t)s, p,
                                    (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long b1 = ((unsigned long long)w.x[1] << 32) | w.x[0];
    const unsigned long long b2 = ((unsigned long long)w.x[3] << 32) | w.x[2];
    const double u1 = (double)(b1 >> 11) * 0x1p-53 + 0x1p-54;
    const double u2 = (double)(b2 >> 11) * 0x1p-53 + 0x1p-54;
    const double r = sqrt(-2.0 * log(u1)) * sd * 0.70710678118654752440;
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    return make_double2(r * cs, r * sn);
}
__device__ __forceinline__ float2 pair_value(uint64_t seed, long long m, int s, uint32_t p, double sd, float)
{
    const Philox4 w = philox4x32_10((uint32_t)m, (uint32_t)((unsigned long long)m >> 32), (uint32_t)s, p,
                                    (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long b1 = ((unsigned long long)w.x[1] << 32) | w.x[0];
    const unsigned long long b2 = ((unsigned long long)w.x[3] << 32) | w.x[2];
    const float u1 = (float)((double)(b1 >> 11) * 0x1p-53 + 0x1p-54);
    const float u2 = (float)((double)(b2 >> 11) * 0x1p-53 + 0x1p-54);
    const float r = sqrtf(-2.0f * logf(u1)) * (float)sd * 0.70710678f;
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    return make_float2(r * cs, r * sn);
}

template <typename T, typename V>
__global__ void sample_kernel(const double *__restrict__ n, int N, uint64_t seed, long long first, long long M,
                              V *__restrict__ rho)
{
    const long long total = M * 2LL * N * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % N);
        const int i = (int)((idx / N) % N);
        const int s = (int)((idx / ((long long)N * N)) % 2);
        const long long mm = idx / (2LL * N * N);
        const double *ns = n + s * N;
        V v;
        if (i == j) {
            v.x = (T)(ns[i] - 0.5);
            v.y = T(0);
        } else {
            const int a = i < j ? i : j, b = i < j ? j : i;
            const uint32_t p = (uint32_t)(a * N - a * (a + 1) / 2 + (b - a - 1));
            const double var = 0.5 * (ns[a] + ns[b] - 2.0 * ns[a] * ns[b]);
            const double sd = var > 0.0 ? sqrt(var) : 0.0;
            v = pair_value(seed, first + mm, s, p, sd, T());
            if (i > j) v.y = -v.y;
        }
        rho[idx] = v;
    }
}

__global__ void philox_kernel(uint64_t seed, long long m, int spin, long long p0, long long count, uint32_t *out)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
         q += (long long)gridDim.x * blockDim.x) {
        const Philox4 w = philox4x32_10((uint32_t)m, (uint32_t)((unsigned long long)m >> 32), (uint32_t)spin,
                                        (uint32_t)(p0 + q), (uint32_t)seed, (uint32_t)(seed >> 32));
        for (int k = 0; k < 4; ++k) out[4 * q + k] = w.x[k];
    }
}

static int grid_for(long long total)
{
    long long g = (total + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 65535LL * 8 ? 65535LL * 8 : g));
}

int launch_sample_diag(Plan *p, const double *occ, uint64_t seed, int64_t first, int64_t M, void *rho,
                       cudaStream_t s)
{
    if (M == 0) return FTWA_OK;
    const long long total = M * 2LL * p->N * p->N;
    if (p->precision == FTWA_FP64)
        sample_kernel<double, double2><<<grid_for(total), 256, 0, s>>>(occ, p->N, seed, first, M,
                                                                      reinterpret_cast<double2 *>(rho));
    else
        sample_kernel<float, float2><<<grid_for(total), 256, 0, s>>>(occ, p->N, seed, first, M,
                                                                    reinterpret_cast<float2 *>(rho));
    return set_cuda_error(cudaGetLastError());
}

// Diagonal initial state: Eq. 7 with the site occupations.  General state
// n = V diag(lambda) V^dagger: Eq. 7 with the eigen-occupations lambda in the
// diagonalising basis, then rho = V rho~ V^dagger (ftwa_basis.cu).
int launch_sample(Plan *p, uint64_t seed, int64_t first, int64_t M, void *rho, cudaStream_t s)
{
    if (!p->general_basis) return launch_sample_diag(p, p->d_n, seed, first, M, rho, s);
    const int rc = launch_sample_diag(p, p->d_lam, seed, first, M, rho, s);
    if (rc != FTWA_OK) return rc;
    return launch_rotate(p, rho, M, s);
}

int launch_philox(uint64_t seed, int64_t m, int32_t spin, int64_t p0, int64_t count, uint32_t *out, cudaStream_t s)
{
    if (count == 0) return FTWA_OK;
    philox_kernel<<<grid_for(count), 256, 0, s>>>(seed, m, spin, p0, count, out);
    return set_cuda_error(cudaGetLastError());
}

}  // namespace ftwa
