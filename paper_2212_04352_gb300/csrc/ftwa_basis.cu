// General (non-diagonal) initial states (App. A, covariance of the Gaussian
// Wigner density; Eq. 7 in a diagonalising basis).
//
// A one-body initial state with density matrix n (per spin, Hermitian,
// eigenvalues in [0, 1]) is given by its eigen-decomposition
// n = V diag(lambda) V^dagger.  In the basis of V the state is diagonal, so
// Eq. 7 applies there with the eigen-occupations lambda; the sample is then
// rotated back, rho = V rho~ V^dagger.  The mean is n - 1/2 and the
// off-diagonal eigen-modes carry the covariance of App. A; as in Eq. 7 the
// diagonal of rho~ carries no noise.
//
// The rotation is two batched complex GEMMs per sample and spin,
// T = rho~ V^dagger and rho = V T, on the CUDA cores in the plan's precision
// (8 N^3 flop each), over chunks of samples whose T fits a 256 MB workspace.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ftwa_internal.h"

namespace ftwa {

namespace rot {

constexpr int kTileR = 64;   // output tile edge
constexpr int kTileK = 16;   // K step

__device__ __forceinline__ void cmad(double2 a, double2 b, double2 &c)
{
    c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
}
__device__ __forceinline__ void cmad(float2 a, float2 b, float2 &c)
{
    c.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x));
    c.y = fmaf(a.x, b.y, fmaf(a.y, b.x, c.y));
}

// One 64 x 64 output tile of C = A B for batch entry z = 2 * (sample) + spin.
//   MODE 0:  A = X[z], B = V[spin]^dagger  (T = rho~ V^dagger)
//   MODE 1:  A = V[spin], B = X[z]         (rho = V T)
// All matrices N x N, row-major, complex.  256 threads, 4 x 4 outputs each
// (rows ty + 16 i, columns tx + 16 j).
template <typename V, int MODE>
__global__ void __launch_bounds__(256) rot_kernel(const V *__restrict__ X, const V *__restrict__ Vb,
                                                  V *__restrict__ Y, int N)
{
    __shared__ V As[kTileK][kTileR + 1];
    __shared__ V Bs[kTileK][kTileR];
    const long long z = blockIdx.z;
    const int s = (int)(z & 1);
    const long long nn = (long long)N * N;
    const V *Xz = X + z * nn;
    const V *Vs = Vb + s * nn;
    const int r0 = blockIdx.y * kTileR, c0 = blockIdx.x * kTileR;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    V acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j].x = 0;
            acc[i][j].y = 0;
        }
    for (int k0 = 0; k0 < N; k0 += kTileK) {
        // A tile: As[kk][rr] = A[r0 + rr][k0 + kk]
        for (int t = threadIdx.x; t < kTileK * kTileR; t += 256) {
            const int kk = t % kTileK, rr = t / kTileK;
            const int r = r0 + rr, k = k0 + kk;
            V a;
            a.x = 0;
            a.y = 0;
            if (r < N && k < N) a = MODE == 0 ? Xz[(long long)r * N + k] : Vs[(long long)r * N + k];
            As[kk][rr] = a;
        }
        // B tile: Bs[kk][cc] = B[k0 + kk][c0 + cc]
        for (int t = threadIdx.x; t < kTileK * kTileR; t += 256) {
            int kk, cc;
            if (MODE == 0) {   // B[k][c] = conj(V[c][k]): read along k
                kk = t % kTileK;
                cc = t / kTileK;
            } else {           // B[k][c] = X[k][c]: read along c
                cc = t % kTileR;
                kk = t / kTileR;
            }
            const int k = k0 + kk, c = c0 + cc;
            V b;
            b.x = 0;
            b.y = 0;
            if (k < N && c < N) {
                if (MODE == 0) {
                    b = Vs[(long long)c * N + k];
                    b.y = -b.y;
                } else {
                    b = Xz[(long long)k * N + c];
                }
            }
            Bs[kk][cc] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTileK; ++kk) {
            V a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cmad(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    V *Yz = Y + z * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= N) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c < N) Yz[(long long)r * N + c] = acc[i][j];
        }
    }
}

}  // namespace rot

void free_basis(Plan *p)
{
    cudaFree(p->d_lam);
    cudaFree(p->d_V);
    cudaFree(p->d_rot_ws);
    p->d_lam = nullptr;
    p->d_V = nullptr;
    p->d_rot_ws = nullptr;
    p->rot_ws_bytes = 0;
    p->general_basis = false;
}

template <typename V>
static int rotate_t(Plan *p, void *rho, int64_t M, cudaStream_t s)
{
    const int N = p->N;
    const size_t per_sample = 2 * (size_t)N * N * sizeof(V);
    const long long chunk = std::max<long long>(1, std::min<long long>(M, (256ll << 20) / (long long)per_sample));
    if (chunk > 32767) return FTWA_ERR_UNSUPPORTED;   // grid z = 2 * chunk
    const size_t need = per_sample * (size_t)chunk;
    if (p->rot_ws_bytes < need) {
        cudaFree(p->d_rot_ws);
        p->d_rot_ws = nullptr;
        p->rot_ws_bytes = 0;
        cudaError_t e = cudaMalloc(&p->d_rot_ws, need);
        if (e != cudaSuccess) return set_cuda_error(e);
        p->rot_ws_bytes = need;
    }
    V *x = reinterpret_cast<V *>(rho);
    V *t = reinterpret_cast<V *>(p->d_rot_ws);
    const V *vb = reinterpret_cast<const V *>(p->d_V);
    const int nt = (N + rot::kTileR - 1) / rot::kTileR;
    for (long long m0 = 0; m0 < M; m0 += chunk) {
        const long long c = std::min<long long>(chunk, M - m0);
        V *xc = x + m0 * 2 * (long long)N * N;
        dim3 grid(nt, nt, (unsigned)(2 * c));
        rot::rot_kernel<V, 0><<<grid, 256, 0, s>>>(xc, vb, t, N);
        rot::rot_kernel<V, 1><<<grid, 256, 0, s>>>(t, vb, xc, N);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    return FTWA_OK;
}

int launch_rotate(Plan *p, void *rho, int64_t M, cudaStream_t s)
{
    if (M == 0) return FTWA_OK;
    return p->precision == FTWA_FP64 ? rotate_t<double2>(p, rho, M, s) : rotate_t<float2>(p, rho, M, s);
}

}  // namespace ftwa

using namespace ftwa;

extern "C" int ftwa_set_initial_basis(ftwa_plan_t *p, const double *lambda, const double *v_re, const double *v_im)
{
    if (!p) return FTWA_ERR_INVALID_ARGUMENT;
    if (!lambda) {
        free_basis(p);
        return FTWA_OK;
    }
    if (!v_re) return FTWA_ERR_INVALID_ARGUMENT;
    const int N = p->N;
    const size_t nn = (size_t)N * N;
    for (int i = 0; i < 2 * N; ++i)
        if (!(lambda[i] >= 0.0 && lambda[i] <= 1.0)) return FTWA_ERR_INVALID_ARGUMENT;
    // V unitary per spin: max |(V^dagger V - 1)_ij| <= 1e-10
    for (int s = 0; s < 2; ++s) {
        const double *re = v_re + s * nn;
        const double *im = v_im ? v_im + s * nn : nullptr;
        for (size_t k = 0; k < nn; ++k)
            if (!std::isfinite(re[k]) || (im && !std::isfinite(im[k]))) return FTWA_ERR_INVALID_ARGUMENT;
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) {
                double gr = 0.0, gi = 0.0;
                for (int k = 0; k < N; ++k) {
                    const double ar = re[(size_t)k * N + i], ai = im ? im[(size_t)k * N + i] : 0.0;
                    const double br = re[(size_t)k * N + j], bi = im ? im[(size_t)k * N + j] : 0.0;
                    gr += ar * br + ai * bi;   // conj(a) b
                    gi += ar * bi - ai * br;
                }
                if (std::fabs(gr - (i == j ? 1.0 : 0.0)) > 1e-10 || std::fabs(gi) > 1e-10)
                    return FTWA_ERR_INVALID_ARGUMENT;
            }
    }
    free_basis(p);
    cudaError_t e = cudaMalloc(&p->d_lam, sizeof(double) * 2 * N);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_lam, lambda, sizeof(double) * 2 * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        if (p->precision == FTWA_FP64) {
            std::vector<double2> h(2 * nn);
            for (size_t k = 0; k < 2 * nn; ++k) h[k] = make_double2(v_re[k], v_im ? v_im[k] : 0.0);
            e = cudaMalloc(&p->d_V, sizeof(double2) * h.size());
            if (e == cudaSuccess) e = cudaMemcpy(p->d_V, h.data(), sizeof(double2) * h.size(), cudaMemcpyHostToDevice);
        } else {
            std::vector<float2> h(2 * nn);
            for (size_t k = 0; k < 2 * nn; ++k) h[k] = make_float2((float)v_re[k], v_im ? (float)v_im[k] : 0.0f);
            e = cudaMalloc(&p->d_V, sizeof(float2) * h.size());
            if (e == cudaSuccess) e = cudaMemcpy(p->d_V, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        free_basis(p);
        return set_cuda_error(e);
    }
    p->general_basis = true;
    return FTWA_OK;
}
