// Sample-mean estimators of Eqs. 5 and 10 from diagonal snapshots.
//
//   mu[t][k]   = (1/M) sum_m X[t][m][k]                 (FP64 snapshots: double,
//                fixed order; FP32 snapshots: 64-bit fixed point, exact to 2^-44)
//   occ[t][k]  = mu + 1/2                               (Eq. 5, first line)
//   conn[t]    = (1/M) (X - mu)^T (X - mu)              (connected Gram)
//   g2[t][k][l] = (conn_kl + occ_k occ_l) / (occ_k occ_l)   (Eq. 10: the sample
//                mean of (X_k + 1/2)(X_l + 1/2) equals conn_kl + occ_k occ_l)
//
// Two Gram paths: FP64 on the CUDA cores (reference), and BF16x3 split
// products on the tcgen05 tensor cores (ftwa_gram_tc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ftwa_internal.h"

namespace ftwa {

// mean over samples, one block per (t, 32-column group); deterministic order
template <typename T>
__global__ void mean_kernel(const T *__restrict__ X, long long M, int K, double *__restrict__ mu,
                            double *__restrict__ occ)
{
    const int t = blockIdx.y;
    const int k = blockIdx.x * 32 + (threadIdx.x & 31);
    const int row = threadIdx.x >> 5;      // 8 row groups
    __shared__ double part[8][32];
    double s = 0.0;
    if (k < K) {
        const T *x = X + (long long)t * M * K + k;
        for (long long m = row; m < M; m += 8) s += (double)x[m * K];
    }
    part[row][threadIdx.x & 31] = s;
    __syncthreads();
    if (row == 0 && k < K) {
        double a = 0.0;
        for (int r = 0; r < 8; ++r) a += part[r][threadIdx.x];
        a /= (double)M;
        mu[t * K + k] = a;
        occ[t * K + k] = a + 0.5;
    }
}

// Sample sums of FP32 snapshots in 64-bit fixed point (units of 2^-44).
// Every FP32 value with |x| < 4 is rounded once, to within 2^-44, and the
// integer additions are exact and associative: the mean is exact to 2^-44
// whatever the order or split of the samples, without one FP64 operation (or
// 64-bit conversion, which runs at FP64 rate on this part) per value.  The
// rounding uses FP32 additions of "magic" constants 1.5 * 2^(23 - s): the
// sum's ulp is 2^-s, so its bit pattern minus the constant's is round(x 2^s):
//   a1 = round(x 2^20)               (x + 12, in [8, 16))
//   r1 = x - a1 2^-20                (exact, |r1| <= 2^-21)
//   a2 = round(r1 2^43)              (r1 + 1.5 2^-20, in [2^-20, 2^-19])
//   x 2^44 ~ a1 2^24 + 2 a2.
// A block that meets |x| >= 4 or a non-finite value marks its partial; the
// final kernel then sums that column in FP64.
constexpr int kMeanRows = 4096;                        // samples per partial
constexpr long long kMeanBad = (long long)(1ULL << 63);   // marker: sum this column in FP64

__device__ __forceinline__ void fx_split(float x, int &a1, int &a2)
{
    const float c1 = 12.0f, c2 = 0x1.8p-20f;
    const float t1 = x + c1;
    a1 = __float_as_int(t1) - __float_as_int(c1);
    const float r1 = x - (t1 - c1);
    const float t2 = r1 + c2;
    a2 = __float_as_int(t2) - __float_as_int(c2);
}

// one block per (32 columns, 4096-sample chunk, time); warp w takes rows
// w, w + 8, ...; eight rows per step in flight, summed in 32 bits per step
__global__ void __launch_bounds__(256) mean_fx_partial_kernel(const float *__restrict__ X, long long M, int K,
                                                              long long *__restrict__ part)
{
    const int t = blockIdx.z, chunk = blockIdx.y, n_chunks = gridDim.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    __shared__ long long sp[8][32];
    __shared__ int sb[8][32];
    long long s1 = 0, s2 = 0;
    int bad = 0;
    if (k < K) {
        const long long m0 = (long long)chunk * kMeanRows;
        const long long m1 = M < m0 + kMeanRows ? M : m0 + kMeanRows;
        const float *x = X + (long long)t * M * K + k;
        long long m = m0 + w;
        for (; m + 56 < m1; m += 64) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = x[(m + 8 * j) * K];
            int b1 = 0, b2 = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                bad |= !(fabsf(v[j]) < 4.0f);
                int a1, a2;
                fx_split(v[j], a1, a2);
                b1 += a1;
                b2 += a2;
            }
            s1 += b1;
            s2 += b2;
        }
        for (; m < m1; m += 8) {
            const float v = x[m * K];
            bad |= !(fabsf(v) < 4.0f);
            int a1, a2;
            fx_split(v, a1, a2);
            s1 += a1;
            s2 += a2;
        }
    }
    sp[w][lane] = s1 * (1LL << 24) + 2 * s2;
    sb[w][lane] = bad;
    __syncthreads();
    if (w == 0 && k < K) {
        long long s_ = 0;
        int b = 0;
        for (int r = 0; r < 8; ++r) {
            s_ += sp[r][lane];
            b |= sb[r][lane];
        }
        part[((long long)t * n_chunks + chunk) * K + k] = b ? kMeanBad : s_;
    }
}

__global__ void mean_fx_final_kernel(const long long *__restrict__ part, int n_chunks, const float *__restrict__ X,
                                     long long M, int K, int T, double *__restrict__ mu, double *__restrict__ occ)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)T * K) return;
    const int t = (int)(i / K), k = (int)(i % K);
    __int128 s = 0;
    bool bad = false;
    for (int c = 0; c < n_chunks; ++c) {
        const long long v = part[((long long)t * n_chunks + c) * K + k];
        if (v == kMeanBad) bad = true;
        s += v;
    }
    double m;
    if (!bad) {
        m = (double)s * 0x1p-44 / (double)M;
    } else {
        double a = 0.0;
        const float *x = X + (long long)t * M * K + k;
        for (long long j = 0; j < M; ++j) a += (double)x[j * K];
        m = a / (double)M;
    }
    mu[i] = m;
    occ[i] = m + 0.5;
}

// FP64 connected Gram: one block per (t, 64x64 tile of the upper triangle);
// 256 threads, 4x4 outputs each; centred samples staged through shared memory.
template <typename T>
__global__ void gram_fp64_kernel(const T *__restrict__ X, long long M, int K, const double *__restrict__ mu,
                                 double *__restrict__ conn, double *__restrict__ g2)
{
    const int t = blockIdx.z;
    const int tk = blockIdx.y, tl = blockIdx.x;
    if (tl < tk) return;
    __shared__ double xa[32][64 + 1];
    __shared__ double xb[32][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    const T *x = X + (long long)t * M * K;
    const double *mut = mu + (long long)t * K;
    for (long long m0 = 0; m0 < M; m0 += 32) {
        for (int i = threadIdx.x; i < 32 * 64; i += 256) {
            const int r = i / 64, c = i % 64;
            const long long m = m0 + r;
            const int ka = tk * 64 + c, kb = tl * 64 + c;
            xa[r][c] = (m < M && ka < K) ? (double)x[m * K + ka] - mut[ka] : 0.0;
            xb[r][c] = (m < M && kb < K) ? (double)x[m * K + kb] - mut[kb] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < 32; ++r) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = xa[r][ty * 4 + i];
                b[i] = xb[r][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    const double inv = 1.0 / (double)M;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const int k = tk * 64 + ty * 4 + i, l = tl * 64 + tx * 4 + j;
            if (k >= K || l >= K) continue;
            const double c = acc[i][j] * inv;
            const double ok = mut[k] + 0.5, ol = mut[l] + 0.5;
            const long long base = (long long)t * K * K;
            conn[base + (long long)k * K + l] = c;
            conn[base + (long long)l * K + k] = c;
            if (g2) {
                const double g = (c + ok * ol) / (ok * ol);
                g2[base + (long long)k * K + l] = g;
                g2[base + (long long)l * K + k] = g;
            }
        }
}

int launch_gram_bf16x3(Plan *p, const void *snap, int64_t M, int32_t T, const double *mu, double *conn,
                       double *g2, cudaStream_t s);
size_t gram_bf16x3_workspace(Plan *p, const void *snap, int64_t M, int32_t T);

static int ensure_workspace(Plan *p, size_t bytes)
{
    if (p->ws_bytes >= bytes) return FTWA_OK;
    if (p->d_ws) cudaFree(p->d_ws);
    p->d_ws = nullptr;
    p->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&p->d_ws, bytes);
    if (e != cudaSuccess) return set_cuda_error(e);
    p->ws_bytes = bytes;
    return FTWA_OK;
}

int launch_moments(Plan *p, const void *snap, int64_t M, int32_t T, double *occ, double *conn, double *g2,
                   int32_t mode, cudaStream_t s)
{
    const int K = 2 * p->N;
    if (mode == FTWA_GRAM_BF16X3 && p->precision != FTWA_FP32) return FTWA_ERR_UNSUPPORTED;
    // workspace: mu [T][K] doubles, then (used in turn) the fixed-point
    // partial sums of the mean and the tensor-core Gram's operands
    const size_t mu_bytes = ((sizeof(double) * (size_t)T * K + 255) / 256) * 256;
    const long long n_chunks = (M + kMeanRows - 1) / kMeanRows;
    if (n_chunks > 65535 || T > 65535) return FTWA_ERR_UNSUPPORTED;
    size_t need = mu_bytes;
    if (p->precision == FTWA_FP32) need += sizeof(long long) * (size_t)T * n_chunks * K;
    if (mode == FTWA_GRAM_BF16X3) need = std::max(need, gram_bf16x3_workspace(p, snap, M, T));
    int rc = ensure_workspace(p, need);
    if (rc != FTWA_OK) return rc;
    double *mu = reinterpret_cast<double *>(p->d_ws);
    if (p->precision == FTWA_FP64) {
        dim3 gm((K + 31) / 32, T);
        mean_kernel<double><<<gm, 256, 0, s>>>(reinterpret_cast<const double *>(snap), M, K, mu, occ);
    } else {
        long long *part = reinterpret_cast<long long *>(reinterpret_cast<unsigned char *>(p->d_ws) + mu_bytes);
        dim3 gm((K + 31) / 32, (unsigned)n_chunks, T);
        mean_fx_partial_kernel<<<gm, 256, 0, s>>>(reinterpret_cast<const float *>(snap), M, K, part);
        rc = set_cuda_error(cudaGetLastError());
        if (rc != FTWA_OK) return rc;
        const long long tk = (long long)T * K;
        mean_fx_final_kernel<<<(unsigned)((tk + 255) / 256), 256, 0, s>>>(part, (int)n_chunks,
                                                                          reinterpret_cast<const float *>(snap), M, K,
                                                                          T, mu, occ);
    }
    rc = set_cuda_error(cudaGetLastError());
    if (rc != FTWA_OK) return rc;
    if (mode == FTWA_GRAM_BF16X3) return launch_gram_bf16x3(p, snap, M, T, mu, conn, g2, s);
    const int nt = (K + 63) / 64;
    dim3 gg(nt, nt, T);
    if (p->precision == FTWA_FP64)
        gram_fp64_kernel<double><<<gg, 256, 0, s>>>(reinterpret_cast<const double *>(snap), M, K, mu, conn, g2);
    else
        gram_fp64_kernel<float><<<gg, 256, 0, s>>>(reinterpret_cast<const float *>(snap), M, K, mu, conn, g2);
    return set_cuda_error(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free moments (ftwa_moments_noalloc).
//
// For callers that cannot call cudaMalloc: applications whose device memory
// is owned by another allocator (a framework's caching allocator or a pool
// sized at start-up) and latency-critical loops that cannot accept
// cudaMalloc's implicit device synchronisation.  The only scratch the FP64
// estimators need, the per-time sample means, lives in the file-scope device
// array below (FTWA_MOMENTS_NOALLOC_MAX_TK doubles, 1 MiB, resident on every
// device that loads the library until the process exits).  Host code must
// not use the array's name as a device address: its device address is looked
// up with cudaGetSymbolAddress with the calling device current.  The lookup
// is repeated on every call whose stream is not capturing, so a device reset
// (which gives the array a new address in the new context) or a switch of
// the current context between calls is picked up; a call on a capturing
// stream reuses the address found by the last non-capturing call on that
// device, which is why a first call must precede any stream capture.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_mu[FTWA_MOMENTS_NOALLOC_MAX_TK];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_lock;
double *g_noalloc_addr[kNoallocMaxDevices] = {nullptr};
}  // namespace

}  // namespace ftwa

extern "C" int ftwa_moments_noalloc(const void *snap_dev, int32_t precision, int32_t n_sites, int64_t M,
                                    int32_t n_times, double *occ_dev, double *conn_dev, double *g2_dev, void *stream)
{
    using namespace ftwa;
    if (!snap_dev || !occ_dev || !conn_dev || M < 1 || n_times < 1 || n_sites < 1 || n_sites > FTWA_MAX_SITES)
        return FTWA_ERR_INVALID_ARGUMENT;
    if (precision != FTWA_FP64 && precision != FTWA_FP32) return FTWA_ERR_INVALID_ARGUMENT;
    const int K = 2 * n_sites;
    if ((int64_t)n_times * K > FTWA_MOMENTS_NOALLOC_MAX_TK) return FTWA_ERR_UNSUPPORTED;
    if (n_times > 65535) return FTWA_ERR_UNSUPPORTED;   // grid y / z extent of the two kernels
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FTWA_ERR_CUDA;
    if (dev < 0 || dev >= kNoallocMaxDevices) return FTWA_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return FTWA_ERR_CUDA;
    double *mu = nullptr;
    {
        std::lock_guard<std::mutex> guard(g_noalloc_lock);
        if (cap == cudaStreamCaptureStatusNone) {
            // fresh lookup: the address belongs to the current context
            void *a = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_mu);
            if (e != cudaSuccess || !a) return FTWA_ERR_CUDA;
            g_noalloc_addr[dev] = static_cast<double *>(a);
        } else if (!g_noalloc_addr[dev]) {
            return FTWA_ERR_UNSUPPORTED;   // no earlier non-capturing call on this device
        }
        mu = g_noalloc_addr[dev];
    }
    // the mean kernel writes every mu[t][k] (t < n_times, k < 2N) before the
    // Gram kernel reads it, so the shared array needs no clearing
    dim3 gm((K + 31) / 32, n_times);
    const int nt = (K + 63) / 64;
    dim3 gg(nt, nt, n_times);
    if (precision == FTWA_FP64) {
        mean_kernel<double><<<gm, 256, 0, s>>>(static_cast<const double *>(snap_dev), M, K, mu, occ_dev);
        gram_fp64_kernel<double><<<gg, 256, 0, s>>>(static_cast<const double *>(snap_dev), M, K, mu, conn_dev, g2_dev);
    } else {
        mean_kernel<float><<<gm, 256, 0, s>>>(static_cast<const float *>(snap_dev), M, K, mu, occ_dev);
        gram_fp64_kernel<float><<<gg, 256, 0, s>>>(static_cast<const float *>(snap_dev), M, K, mu, conn_dev, g2_dev);
    }
    return set_cuda_error(cudaGetLastError());
}

