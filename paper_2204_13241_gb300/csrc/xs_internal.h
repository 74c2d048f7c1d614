// Internal launch interface between the C ABI (xs_api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "xs_common.cuh"

namespace xs {

// Sets the message xs_last_error() returns on the calling thread.
void set_last_error(const char* msg);

// Kernels launched by the calling host thread (each launch_* adds its own);
// the ABI layer turns the deltas into per-context counts.
extern thread_local int64_t tl_kernel_launches;

struct GridDesc {
    int nx0, nx, ny0, ny, nz0, nz;
    __host__ __device__ int64_t pixels() const { return (int64_t)nx * ny * nz; }
};

// ---- phase records (fractional coordinates as 32-bit turns) -------------
// rec [n_frames][n_pad]; the slots hold runs of kPermRun consecutive atoms:
// slot k of a frame holds atom j = kPermRun ((k / kPermRun) perm_mul mod
// n_pad / kPermRun) + k mod kPermRun (perm_mul coprime with n_pad / kPermRun;
// 1 keeps the input order); atoms >= n_atoms get f = 0 and U = 0.  `ortho`:
// h^-1 is diagonal; `need_z`: U_z is used (otherwise it is left 0).
constexpr int64_t kPermRun = 8;
struct PhaseOpts {
    bool ortho = false;
    bool need_z = true;
    int64_t perm_mul = 1;                // permutes the runs of kPermRun atoms
    float lim[3] = {0.0f, 0.0f, 0.0f};  // set by launch_phase
    const int32_t* index = nullptr;      // optional device [n_atoms]: atoms of the frames to use
    int64_t pos_atoms = 0;               // atoms per frame of `pos` when `index` is given
    bool pos8 = false;                   // set by launch_phase: `pos` is 8-byte aligned
    // set by launch_phase for orthorhombic cells: 2^32 h^-1_aa = (-1)^cneg cm 2^ce
    // with cm = ch 2^32 + cl a 53-bit integer
    uint32_t ch[3] = {0, 0, 0}, cl[3] = {0, 0, 0};
    int ce[3] = {0, 0, 0};
    uint32_t cneg[3] = {0, 0, 0};
};
cudaError_t launch_phase(const float* pos, const float* f, int64_t n_atoms, int64_t n_frames,
                         int64_t n_pad, const Mat3& hinv, const PhaseOpts& opt, AtomRec* rec, int* err,
                         cudaStream_t st);
// What the phase kernel needs to build the record of any (frame, slot):
// `opt` completed by make_phase_src, hs = 2^32 h^-1.
struct PhaseSrc {
    const float* pos = nullptr;  // frame 0 of the records: [frames][stride][3]
    const float* f = nullptr;
    int64_t n_atoms = 0;
    int64_t n_pad = 0;
    Mat3 hs;
    PhaseOpts opt;
    AtomRec* rec = nullptr;      // [frames][n_pad]
};
// Completes `opt` for the kernels; false when the permutation's products could
// overflow (perm_mul != 1 with n_pad >= 2^32 or not a multiple of kPermRun)
bool make_phase_src(const float* pos, const float* f, int64_t n_atoms, int64_t n_pad, const Mat3& hinv,
                    const PhaseOpts& opt, AtomRec* rec, PhaseSrc& out);

// ---- plain FP32 direct sum ----------------------------------------------
struct DirectPlan {
    int splits;            // atom splits (partials merged in FP64 by a second kernel)
    int64_t atoms_per_split;
    size_t partial_bytes;  // workspace for the partial amplitudes
};
DirectPlan plan_direct(int64_t n_pad, int64_t n_frames, const GridDesc& g, int num_sms);
// pts (optional, device int32 [P][3]): Miller indices of P arbitrary points;
// g then only gives P as g.nx with ny = nz = 1
cudaError_t launch_direct(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g,
                          const DirectPlan& plan, void* partial, float* I, float* amp,
                          cudaStream_t st, const int32_t* pts = nullptr);

// ---- factorised FP32 direct sum -------------------------------------------
struct FactoredPlan {
    int splits;            // atom ranges (FP64 partial amplitudes added in order by a second kernel)
    int64_t atoms_per_split;
    size_t partial_bytes;  // workspace for the partial amplitudes
};
FactoredPlan plan_factored(int64_t n_pad, int64_t n_frames, const GridDesc& g, int num_sms);
cudaError_t launch_factored(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g,
                            const FactoredPlan& plan, void* partial, float* I, float* amp, cudaStream_t st);

// ---- tensor-core split-precision contraction ----------------------------
// One trajectory of a launch: phase records [n_frames][n_pad] (slot order of
// the phase kernel), outputs, and its grid; tiles are 128 x 128 pixels.
// Tile kinds of the pair contraction: kTcTile128 covers 128 n_x x 128 n_y
// (MMA N = 256, 8 producer warps with runs of 32 n), kTcTile64 covers
// 128 n_x x 64 n_y (MMA N = 128, 12 producer warps with runs of 16 n).
constexpr int kTcTile128 = 0;
constexpr int kTcTile64 = 1;
__host__ __device__ constexpr inline int tc_tile_y(int kind) { return kind == kTcTile64 ? 64 : 128; }  // n_y per tile

struct TcTraj {
    const uint4* rec;
    float* I;
    float* amp;
    int64_t n_pad;
    int n_stages;  // n_pad / 64
    int tiles_x, tiles_y;
    int nx0, nx, ny0, ny, nz0, nz;
    int n_frames;
    int kind;      // tile kind (all trajectories of one launch share it)
    int chunk;     // stages per FP32 accumulation chunk; 0: the launch's
    int exact;     // 1: tables from FP64 sincospi per entry (test and measurement option)
#ifdef XS_BOUNDS_CHECK
    int check_frames;  // frames of I and amp the bounds check admits (n_frames; one less in the self-test)
#endif
};
bool tc_supported(const GridDesc& g);
int64_t tc_atom_multiple();
int tc_pair_capacity(int num_sms, int kind = kTcTile128);  // co-resident CTA pairs
TcTraj tc_traj(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g, float* I, float* amp,
               int kind = kTcTile128, int chunk = 0, bool exact = false);
// tile kind for a (contracted) grid when nothing was tuned: 128 x 64 tiles
// where they need no more tiles than 128 x 128 ones (n_y extent <= 64)
int tc_default_kind(const GridDesc& g);
int64_t tc_units(const TcTraj& t);  // frames x planes x tiles
size_t tc_scratch_bytes(int n_pairs);
// per-pair unit lists (traj, frame, plane, tile_x | tile_y << 16), longest first
// longest-processing-time dealing of explicit units (traj, frame, plane, tile_x | tile_y << 16)
void tc_deal_units(const std::vector<TcTraj>& trajs, const std::vector<int4>& all, int n_pairs,
                   std::vector<int4>& units, std::vector<int>& pair_start);
void tc_build_lists(const std::vector<TcTraj>& trajs, int n_pairs, std::vector<int4>& units,
                    std::vector<int>& pair_start);
// stages (of 64 atoms) per FP32 tensor-core accumulation before the epilogue
// adds the chunk into its TwoSum totals.  The tensor core's FP32 accumulation
// is biased, so the error grows with the chunk: on the 256,000-atom crystal
// e_I is 1.4e-5 at 32 stages and 2.9e-5 at 64, which runs 5% faster.
constexpr int kDefaultChunkStages = 64;

// dealing of a single trajectory's units over the pairs: `full` whole waves,
// then `rem` units cut into `parts` pieces along the atoms (parts = 1: plain
// round-robin of all units, full = 0)
struct TcSplit {
    int64_t full = 0, rem = 0;
    int parts = 1;
};
TcSplit tc_split_plan(int64_t units, int n_pairs, int n_stages, int chunk_stages);
size_t tc_split_bytes(const TcSplit& sp);  // FP64 partial amplitudes of the pieces
cudaError_t launch_tc_single(const TcTraj& tr, int n_pairs, const TcSplit& sp, int chunk_stages, bool bf16,
                             double* scratch, void* split_buf, int* err, int64_t timeout_ns, cudaStream_t st);
// sums the pieces of the split units of a launch_tc_single launch (same
// arguments) into I; run after it on the same stream
cudaError_t launch_tc_split_finish(const TcTraj& tr, int n_pairs, const TcSplit& sp, void* split_buf,
                                   cudaStream_t st);
cudaError_t launch_tc_batch(const TcTraj* d_trajs, const int4* d_units, const int* d_pair_start, int n_pairs,
                            int chunk_stages, bool bf16, int kind, bool exact, double* scratch, int* err,
                            int64_t timeout_ns, cudaStream_t st);

// ---- g2 -----------------------------------------------------------------
int g2_segments(int64_t T);
size_t g2_workspace_bytes(int64_t T, int64_t P, int n_tau);  // FP64 partial sums per frame segment
cudaError_t launch_g2(const float* I, int64_t T, int64_t P, const int32_t* d_taus, int n_tau,
                      double* g2, double* mean, void* ws, cudaStream_t st);

// ---- XSVS contrast --------------------------------------------------------
struct XsvsLayout {
    int64_t n_in_rings;   // pixels that belong to a ring
    int n_chunks;         // (ring, pixel range) chunks
    int64_t n_kw;         // sum over K of floor(T/K)
};
// rows of the XSVS prefix buffer (float64 [rows][pixels in rings]): T + 1
// prefix rows and the frame-segment totals after them
int64_t xsvs_prefix_rows(int64_t T);
// Algorithm 2 grid: n^3 points of an orthorhombic cell, spacing h[a], k[a]
// Gaussian weights per axis around each atom
struct FftGrid {
    int n;
    double h[3];
    int k[3];
    double inv_2eta2;  // 1 / (2 eta^2)
};
cudaError_t launch_fft_frame(const float* pos, const float* f, int64_t n_atoms, const FftGrid& fg, double2* grid,
                             const GridDesc& g, const double2* d_G, float* I, float* amp, int* err, cudaStream_t st);
// grids computed as a half plus mirrors (real form factors: I(-q) = I(q)):
// returns the split axis (0: n_x for planes at n_z = 0, 2: n_z) and the half
// grid v when v needs fewer 128 x 128 tiles than g, else -1
int friedel_half_grid(const GridDesc& g, GridDesc& v);
// I [T][g] (and amp, conjugated where mirrored; NULL to skip) from the half
// [T][v]
cudaError_t launch_friedel(const float* half, const float* half_amp, int64_t T, const GridDesc& v, const GridDesc& g,
                           int axis, float* I, float* amp, cudaStream_t st);
cudaError_t launch_points_gather(const float* tmp, const float* tmp_amp, const int64_t* d_src, const int64_t* d_stride,
                                 int64_t P, int64_t nf, float* I, float* amp, cudaStream_t st);
cudaError_t launch_ff_table(const double* d_coef, int n_species, const GridDesc& g, const Mat3& hinv, double* table,
                            cudaStream_t st);
cudaError_t launch_species_acc(const float* S, const double* ff, int64_t nf, int64_t P, bool first, double* acc,
                               cudaStream_t st);
cudaError_t launch_species_finish(const double* acc, int64_t n, float* I, float* amp, cudaStream_t st);
// XSVS window sums per ring for a pixel subset: sums [n_kw][n_rings] of (sum x, sum x^2)
cudaError_t launch_xsvs_partial(const float* I, int64_t T, int64_t P, const int32_t* d_perm, const int4* d_chunks,
                               int n_chunks, int64_t n_in_rings, const int32_t* d_K, const int64_t* d_kw_off, int n_K,
                               int64_t n_kw, const int32_t* d_ring_first_chunk, int n_rings, double* prefix,
                               double2* partial, double* sums, cudaStream_t st);
cudaError_t launch_isf(const float* amp, int64_t T, int64_t P, const int32_t* d_taus, int n_tau, double inv_sum_f2,
                       double* F, double* Fhat, cudaStream_t st);
cudaError_t launch_isf_contrast(const double* Fhat, int64_t Kmax, int64_t P, const int32_t* d_perm, int64_t n_in,
                                const int32_t* d_K_sorted, const int32_t* d_k_row, int n_K,
                                const int64_t* d_ring_start, int n_rings, double* b_pixel, double* out,
                                cudaStream_t st);
cudaError_t launch_xsvs(const float* I, int64_t T, int64_t P, const int32_t* d_perm,
                        const int4* d_chunks, int n_chunks, int64_t n_in_rings,
                        const int32_t* d_K, const int64_t* d_kw_off, int n_K, int64_t n_kw,
                        const int32_t* d_ring_first_chunk, const int32_t* d_ring_count,
                        int n_rings, double* prefix, double2* partial, double* beta,
                        cudaStream_t st);

// ---- adjoint --------------------------------------------------------------
size_t adjoint_workspace_bytes(const GridDesc& g, int64_t n_pad);
cudaError_t launch_adjoint(const AtomRec* rec, int64_t n_atoms, int64_t n_pad, const GridDesc& g,
                           const Mat3& hinv, const float* amp, const float* dL_dI,
                           void* workspace, float* grad, int* err, int64_t timeout_ns, cudaStream_t st);
// the contraction over n_y on tensor cores (split BF16): the H image, built
// from amp [P][2] and dL/dI [P], and the per-unit partial sums,
// adjoint_tc_image_bytes(g, n_pad) bytes (16-byte aligned)
size_t adjoint_tc_image_bytes(const GridDesc& g, int64_t n_pad);
cudaError_t launch_adjoint_tc(const AtomRec* rec, int64_t n_atoms, int64_t n_pad, const GridDesc& g,
                              const Mat3& hinv, const float* amp, const float* G, void* image, float* grad, int* err,
                              int64_t timeout_ns, cudaStream_t st);

}  // namespace xs
