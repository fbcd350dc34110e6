// Internal declarations shared by the translation units of libftwa.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/ftwa.h"

namespace ftwa {

constexpr int kMaxCluster = 8;
constexpr int kThreads = 768;          // threads per CTA of the stepper
constexpr int kWarps = kThreads / 32;
constexpr int kTmemCols = 512;         // one CTA per SM holds all of tensor memory
// tensor-memory columns of one warp: warps w, w+4, ... share lane quadrant
// w % 4 and split the 512 columns (multiple of 8 for aligned x8 accesses)
constexpr int kTmemColsPerWarp = (kTmemCols / (kWarps / 4)) / 8 * 8;
constexpr int kMinSmem = 120 * 1024;   // forces one stepper CTA per SM

// Launch shape of the RK4 stepper for one slot count.
struct StepperShape {
    int cluster = 1;        // CTAs per sample group
    int slots = 1;          // samples per cluster (cluster == 1 only)
    int units_per_warp = 0; // E: 32-column work units per warp
    int n_units = 0;        // work units of the busiest rank
    int smem_bytes = 0;
    int buf_bytes = 0;      // bytes of one stage buffer (max over ranks)
    int row_begin[kMaxCluster + 1] = {0};  // spin-row partition over ranks
    int grid = 0;           // CTAs launched
    int variant = 0;        // 1 = banded stepper, 2 = general packed-triangle stepper, 3 = tiled stepper
    int threads = kThreads; // threads per CTA
};

// Launch shape of the banded stepper.
struct BandShape {
    int cluster = 1, slots = 1, E = 0, k_items = 0, buf_bytes = 0, smem_bytes = 0, grid = 0;
    int qoff = 0;    // first column of column block 0 (<= 0)
    int row_begin[kMaxCluster + 1] = {0};
    std::vector<uint32_t> items;   // [cluster][kWarps][k_items]
};

struct Plan {
    int device = 0;
    int N = 0, B = 0;
    int precision = FTWA_FP64;
    double U = 0, dt = 0.01;
    int out_every = 10;
    int cluster_override = 0, threads_override = 0, autotune = 0;
    uint64_t timeout_ns = 5000000000ull;
    int force_timeout = 0;
    int sm_count = 0;
    bool uniform_t = true;
    int bandwidth = 1;                // max over bonds of j - i (site ordering)
    std::vector<int32_t> bonds;       // [B][2]
    std::vector<double> t_bond;       // [B]
    std::vector<double> n_up, n_dn;   // [N]
    std::vector<int32_t> nbr_host;    // [N]: k0 | k1 << 8 | k2 << 16 | deg << 24
    std::vector<int32_t> nbr_bond;    // [N][3]: bond index of each slot (-1 if none)
    // device tables
    int32_t *d_nbr = nullptr;         // [N]
    int32_t *d_nbr_bond = nullptr;    // [N][3]
    double *d_t64 = nullptr;          // [N][4] hopping per neighbour slot
    float *d_t32 = nullptr;           // [N][4]
    double *d_n = nullptr;            // [2][N] occupations
    int32_t *d_bonds = nullptr;       // [B][2]
    int *d_status = nullptr;          // device status word
    void *d_ws = nullptr;             // plan-owned workspace (moments, adjoint)
    void *d_adj_ws = nullptr;         // adjoint per-CTA workspace
    size_t adj_ws_bytes = 0;
    void *d_corr_ws = nullptr;        // adjoint: symmetrised correlation cotangents and means
    size_t corr_ws_bytes = 0;
    void *d_tile = nullptr;           // tiled stepper tables (tiles, row-part offsets, hoppings)
    size_t tile_bytes = 0;
    std::vector<unsigned char> tile_host;   // copy of the tables last uploaded
    std::vector<int> tile_rp_k;             // tiled stepper: row-part slot columns (lattice only;
    std::vector<char> tile_rp_real;         //   searched once, empty until the first use)
    std::vector<float> tile_rp_t;
    uint32_t *d_items = nullptr;      // banded stepper work items
    size_t items_bytes = 0;
    std::vector<uint32_t> items_host; // copy of the table last uploaded
    bool dry_run = false;             // choose the shape and upload tables, launch nothing
    int variant_override = 0;         // 0 auto, 1 banded only, 2 general only, 3 tiled only
    size_t ws_bytes = 0;
    StepperShape shape;               // chosen for the full machine
    // general (non-diagonal) initial state n = V diag(lambda) V^dagger per spin
    bool general_basis = false;
    double *d_lam = nullptr;          // [2][N] eigen-occupations lambda
    void *d_V = nullptr;              // [2][N][N] complex eigenvectors (columns), plan precision
    void *d_rot_ws = nullptr;         // rotation workspace (chunk of samples)
    size_t rot_ws_bytes = 0;
    // time-dependent on-site drive v_i,s(t) = amp[s][i] f(t)
    bool drive = false;
    double drive_t0 = 0, drive_sigma = 0, drive_omega = 0, drive_phase = 0;
    double *d_amp64 = nullptr;        // [2][N]
    float *d_amp32 = nullptr;         // [2][N]
    void *d_ftab = nullptr;           // [n_steps][4] pulse values of the last evolve call
    size_t ftab_bytes = 0;
    // time-dependent hopping scale m(t) = 1 + hop_eps g(t)
    bool hop_drive = false;
    double hop_eps = 0, hop_t0 = 0, hop_sigma = 0, hop_omega = 0, hop_phase = 0;
    // long-range interaction u_ij of Eq. 1 (replaces the on-site U)
    bool longrange = false;
    double *d_u64 = nullptr;          // [N][N]
    float *d_u32 = nullptr;           // [N][N]
};

int set_cuda_error(cudaError_t e);

// per-translation-unit launchers
int launch_sample(Plan *p, uint64_t seed, int64_t first, int64_t M, void *rho, cudaStream_t s);
int launch_sample_diag(Plan *p, const double *occ, uint64_t seed, int64_t first, int64_t M, void *rho,
                       cudaStream_t s);
int launch_rotate(Plan *p, void *rho, int64_t M, cudaStream_t s);
void free_basis(Plan *p);
int launch_philox(uint64_t seed, int64_t m, int32_t spin, int64_t p0, int64_t count, uint32_t *out,
                  cudaStream_t s);
int launch_evolve(Plan *p, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s,
                 double t_start = 0.0);
void free_drive(Plan *p);
void free_interaction(Plan *p);
int choose_stepper_shape(Plan *p, int64_t M, StepperShape *out);
bool tile_supported(const Plan *p);
int launch_tile(Plan *p, void *rho, int64_t M, int64_t n_steps, void *snap, cudaStream_t s);
int choose_band_shape(Plan *p, int64_t M, BandShape *out);
int launch_moments(Plan *p, const void *snap, int64_t M, int32_t T, double *occ, double *conn, double *g2,
                   int32_t mode, cudaStream_t s);
int launch_adjoint(Plan *p, uint64_t seed, int64_t M, int64_t n_steps, int32_t ckpt_every, const double *dL,
                   const double *dC, const double *occ, double *gU, double *gt, double *gn, cudaStream_t s);

}  // namespace ftwa

// The opaque handle of the C ABI is the plan itself.
struct ftwa_plan : public ftwa::Plan {};

// A batched launch: one CUDA graph (kernel branches of several plans, or one
// persistent kernel over a work queue of all plans' samples) and the device
// memory the batch owns (work queue, tables).
struct ftwa_batch {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n = 0;
    void *d_owned = nullptr;
};
