// Factorised FP32 direct sum (Algorithm 1 with the factorisation of Sec. 3.1,
// on the FP32 SIMT pipes).
//
// For q on the reciprocal lattice exp(i q.r_j) = E_x[n_x](j) E_y[n_y](j)
// E_z[n_z](j), so one plane of S is the complex contraction over atoms
//   S(n_x, n_y) = sum_j E_x[n_x](j) W_j(n_y),   W_j(n_y) = f_j E_z[n_z](j) E_y[n_y](j).
// fx_kernel: a block of 256 threads owns a tile of 64 n_x by 64 n_y of one
// frame and plane and a range of atoms.  Per stage of 32 atoms it builds the
// tables E_x (32 x 64) and W (32 x 64) in shared memory from FP32 sincospi of
// exact integer turn counts (the arithmetic of the plain direct kernel), a
// seed per run of 4 entries advanced by exp(i 2 pi U), then every thread adds
// E_x W over the stage's atoms into
// its 4 x 4 pixels: one complex multiply-add (4 FP32 FMAs) per
// atom*pixel against the plain kernel's sincospi and compensated update of
// about 53 instructions.  Each stage's 32-term FP32 sums are added into
// running totals kept as error-free FP32 pairs (TwoSum), so the error stays
// that of 32-term sums; with several atom ranges ("splits") the FP64 partial
// amplitudes are added in a fixed order by fx_reduce_kernel.
#include "xs_internal.h"

#include <algorithm>

namespace xs {

namespace {

constexpr int kFxTile = 64;     // n_x and n_y per block
constexpr int kFxAtoms = 32;    // atoms per stage
constexpr int kFxThreads = 256;
constexpr size_t kFxTabBytes = 2 * 2 * kFxAtoms * kFxTile * sizeof(float2);  // E_x and W, two buffers: 64 KB
// plus the low parts of the running totals, [32 values][256 threads] (32 KB):
// kept in shared memory, where they are touched once per stage, instead of
// 32 registers that the inner loop needs
constexpr size_t kFxSmemBytes = kFxTabBytes + 32 * kFxThreads * sizeof(float);

struct FxArgs {
    const AtomRec* rec;
    int64_t n_pad;
    int n_frames;
    GridDesc g;
    int tiles_x, tiles_y;
    int64_t atoms_per_split;  // a multiple of kFxAtoms
    double2* partial;         // [splits][n_frames][P] when splits > 1
    float* I;
    float* amp;
};

__device__ __forceinline__ float2 fx_cis(uint32_t P) {
    float c, s;
    phase_to_cs(P, c, s);
    return make_float2(c, s);
}

// Shared-memory layout of a table row (one atom, 64 complex entries = 512 B):
// four 128-byte lines of 16 entries, each line eight 16-byte chunks of two
// entries.  Chunk c of line l (l = 4 atom + segment) is stored at position
// c ^ (l & 7): a table builder's store instruction has its 32 threads on 32
// lines at the same chunk, which without the swizzle would fall on the same
// banks (32 wavefronts instead of 4), while the readers' loads of one atom
// stay within one line (E_x) or two lines at disjoint positions (W).
__device__ __forceinline__ int fx_slot(int atom, int seg, int chunk) {
    return atom * kFxTile + seg * 16 + 2 * (chunk ^ ((atom * 4 + seg) & 7));
}

// TwoSum: hi + lo += c with the rounding error of hi + c carried in lo
__device__ __forceinline__ void two_sum(float& hi, float* lo, float c) {
    const float s = hi + c;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (c - bb);
    hi = s;
    *lo += e;
}

// grid: x = (frame, plane, tile), y = atom split
__global__ void __launch_bounds__(kFxThreads, 2) fx_kernel(FxArgs a) {
    extern __shared__ __align__(16) float2 fx_smem[];
    auto s_ex = reinterpret_cast<float2(*)[kFxAtoms][kFxTile]>(fx_smem);
    auto s_w = reinterpret_cast<float2(*)[kFxAtoms][kFxTile]>(fx_smem + 2 * kFxAtoms * kFxTile);
    const GridDesc& g = a.g;
    int64_t u = blockIdx.x;
    const int tx = (int)(u % a.tiles_x);
    u /= a.tiles_x;
    const int ty = (int)(u % a.tiles_y);
    u /= a.tiles_y;
    const int iz = (int)(u % g.nz);
    const int t = (int)(u / g.nz);
    const int split = blockIdx.y;
    const int64_t a0 = (int64_t)split * a.atoms_per_split;
    const int64_t a1 = min(a.n_pad, a0 + a.atoms_per_split);
    const AtomRec* frame_rec = a.rec + (int64_t)t * a.n_pad;
    const int x0 = tx * kFxTile, y0 = ty * kFxTile;
    const uint32_t nz = (uint32_t)(g.nz0 + iz);

    const int tid = threadIdx.x;
    // table builder: atom tid / 8 of the stage, 16 consecutive n of E_x
    // (segments 0-3) or of W (segments 4-7)
    const int b_atom = tid >> 3, b_seg = tid & 7;
    // accumulator owner: 4 x 4 pixels, a warp spans 4 x-groups and 8 y-groups
    const int warp = tid >> 5, lane = tid & 31;
    const int xg = (warp & 3) * 4 + (lane & 3);
    const int yg = (warp >> 2) * 8 + (lane >> 2);

    float sr[4][4], si[4][4];     // this stage's sums
    float hr[4][4], hi_[4][4];    // running totals, high parts
    // low parts: value v = 2 (4 x + y) + (0: re, 1: im) of this thread
    float* s_lo = reinterpret_cast<float*>(reinterpret_cast<char*>(fx_smem) + kFxTabBytes) + tid;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            hr[x][y] = hi_[x][y] = 0.0f;
            s_lo[(2 * (4 * x + y)) * kFxThreads] = 0.0f;
            s_lo[(2 * (4 * x + y) + 1) * kFxThreads] = 0.0f;
        }

    int buf = 0;
    for (int64_t k0 = a0; k0 < a1; k0 += kFxAtoms, buf ^= 1) {
        {
            const int64_t j = k0 + b_atom;
            AtomRec r;
            r.ux = r.uy = r.uz = 0u;
            r.f = 0.0f;
            if (j < a1) r = frame_rec[j];
            // 16 entries as 4 runs of 4: an exact seed per run and at most
            // three steps by exp(i 2 pi U), so each entry carries at most
            // three FP32 rotations (about 2e-7) beyond its seed's rounding
            const bool is_x = b_seg < 4;
            const uint32_t U = is_x ? r.ux : r.uy;
            const uint32_t n0 = is_x ? (uint32_t)(g.nx0 + x0 + 16 * b_seg) : (uint32_t)(g.ny0 + y0 + 16 * (b_seg - 4));
            float2 wz = make_float2(1.0f, 0.0f);
            if (!is_x) {
                wz = make_float2(r.f, 0.0f);
                if (nz != 0u) {
                    const float2 ez = fx_cis(nz * r.uz);
                    wz = make_float2(r.f * ez.x, r.f * ez.y);
                }
            }
            const float2 z = fx_cis(U);
            float2* row = is_x ? &s_ex[buf][0][0] : &s_w[buf][0][0];
            const int seg = b_seg & 3;
#pragma unroll
            for (int run = 0; run < 4; ++run) {
                const float2 e0 = fx_cis((n0 + 4u * (uint32_t)run) * U);
                float2 e = make_float2(fmaf(e0.x, wz.x, -e0.y * wz.y), fmaf(e0.x, wz.y, e0.y * wz.x));
                float4 v01, v23;
                v01.x = e.x;
                v01.y = e.y;
                e = make_float2(fmaf(e.x, z.x, -e.y * z.y), fmaf(e.x, z.y, e.y * z.x));
                v01.z = e.x;
                v01.w = e.y;
                e = make_float2(fmaf(e.x, z.x, -e.y * z.y), fmaf(e.x, z.y, e.y * z.x));
                v23.x = e.x;
                v23.y = e.y;
                e = make_float2(fmaf(e.x, z.x, -e.y * z.y), fmaf(e.x, z.y, e.y * z.x));
                v23.z = e.x;
                v23.w = e.y;
                *reinterpret_cast<float4*>(row + fx_slot(b_atom, seg, 2 * run)) = v01;
                *reinterpret_cast<float4*>(row + fx_slot(b_atom, seg, 2 * run + 1)) = v23;
            }
        }
        __syncthreads();  // the tables of this stage are complete; the other buffer's readers are done
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) sr[x][y] = si[x][y] = 0.0f;
#pragma unroll 4
        for (int k = 0; k < kFxAtoms; ++k) {
            // entries 4 xg .. 4 xg + 3: chunks 2 (xg & 3), +1 of line segment xg >> 2
            const float2* ex = &s_ex[buf][0][0];
            const float2* wy = &s_w[buf][0][0];
            const float4 e01 = *reinterpret_cast<const float4*>(ex + fx_slot(k, xg >> 2, 2 * (xg & 3)));
            const float4 e23 = *reinterpret_cast<const float4*>(ex + fx_slot(k, xg >> 2, 2 * (xg & 3) + 1));
            const float4 w01 = *reinterpret_cast<const float4*>(wy + fx_slot(k, yg >> 2, 2 * (yg & 3)));
            const float4 w23 = *reinterpret_cast<const float4*>(wy + fx_slot(k, yg >> 2, 2 * (yg & 3) + 1));
            const float ex_r[4] = {e01.x, e01.z, e23.x, e23.z}, ex_i[4] = {e01.y, e01.w, e23.y, e23.w};
            const float w_r[4] = {w01.x, w01.z, w23.x, w23.z}, w_i[4] = {w01.y, w01.w, w23.y, w23.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    sr[x][y] = fmaf(ex_r[x], w_r[y], fmaf(-ex_i[x], w_i[y], sr[x][y]));
                    si[x][y] = fmaf(ex_r[x], w_i[y], fmaf(ex_i[x], w_r[y], si[x][y]));
                }
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                two_sum(hr[x][y], &s_lo[(2 * (4 * x + y)) * kFxThreads], sr[x][y]);
                two_sum(hi_[x][y], &s_lo[(2 * (4 * x + y) + 1) * kFxThreads], si[x][y]);
            }
    }

    const int64_t P = g.pixels();
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int ix = x0 + 4 * xg + x;
        if (ix >= g.nx) continue;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int iy = y0 + 4 * yg + y;
            if (iy >= g.ny) continue;
            const double re = (double)hr[x][y] + (double)s_lo[(2 * (4 * x + y)) * kFxThreads];
            const double im = (double)hi_[x][y] + (double)s_lo[(2 * (4 * x + y) + 1) * kFxThreads];
            const int64_t p = ((int64_t)iz * g.ny + iy) * g.nx + ix;
            if (gridDim.y > 1) {
                a.partial[((int64_t)split * a.n_frames + t) * P + p] = make_double2(re, im);
            } else {
                const int64_t o = (int64_t)t * P + p;
                a.I[o] = (float)(re * re + im * im);
                if (a.amp) {
                    a.amp[2 * o] = (float)re;
                    a.amp[2 * o + 1] = (float)im;
                }
            }
        }
    }
}

// one thread per (frame, pixel): the splits' partial amplitudes in split order
__global__ void fx_reduce_kernel(const double2* __restrict__ partial, int splits, int64_t n_items,
                                 float* __restrict__ I, float* __restrict__ amp) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items;
         i += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int s = 0; s < splits; ++s) {
            const double2 v = partial[(int64_t)s * n_items + i];
            re += v.x;
            im += v.y;
        }
        I[i] = (float)(re * re + im * im);
        if (amp) {
            amp[2 * i] = (float)re;
            amp[2 * i + 1] = (float)im;
        }
    }
}

}  // namespace

FactoredPlan plan_factored(int64_t n_pad, int64_t n_frames, const GridDesc& g, int num_sms) {
    FactoredPlan p;
    const int64_t tiles = ((int64_t)(g.nx + kFxTile - 1) / kFxTile) * ((g.ny + kFxTile - 1) / kFxTile) * g.nz;
    const int64_t blocks = tiles * n_frames;
    const int64_t stages = (n_pad + kFxAtoms - 1) / kFxAtoms;
    // enough blocks for four per SM, each with at least 8 stages of atoms
    int64_t splits = std::max<int64_t>(1, (4 * (int64_t)num_sms + blocks - 1) / std::max<int64_t>(blocks, 1));
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, stages / 8));
    splits = std::min<int64_t>(splits, 65535);
    const int64_t st_per = (stages + splits - 1) / splits;
    p.atoms_per_split = st_per * kFxAtoms;
    p.splits = (int)((n_pad + p.atoms_per_split - 1) / p.atoms_per_split);
    p.partial_bytes = p.splits > 1 ? (size_t)p.splits * n_frames * g.pixels() * sizeof(double2) : 0;
    return p;
}

cudaError_t launch_factored(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g,
                            const FactoredPlan& plan, void* partial, float* I, float* amp, cudaStream_t st) {
    const int64_t P = g.pixels();
    if (P == 0 || n_frames == 0) return cudaSuccess;
    FxArgs a;
    a.rec = rec;
    a.n_pad = n_pad;
    a.n_frames = (int)n_frames;
    a.g = g;
    a.tiles_x = (g.nx + kFxTile - 1) / kFxTile;
    a.tiles_y = (g.ny + kFxTile - 1) / kFxTile;
    a.atoms_per_split = plan.atoms_per_split;
    a.partial = static_cast<double2*>(partial);
    a.I = I;
    a.amp = amp;
    const int64_t blocks = (int64_t)a.tiles_x * a.tiles_y * g.nz * n_frames;
    if (blocks > INT32_MAX || plan.splits > 65535) return cudaErrorInvalidValue;
    if (plan.splits > 1 && !partial) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFxSmemBytes);
    if (e != cudaSuccess) return e;
    ++tl_kernel_launches;
    fx_kernel<<<dim3((unsigned)blocks, (unsigned)plan.splits), kFxThreads, kFxSmemBytes, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess || plan.splits <= 1) return e;
    const int64_t items = n_frames * P;
    ++tl_kernel_launches;
    fx_reduce_kernel<<<(unsigned)std::min<int64_t>((items + 255) / 256, 65535), 256, 0, st>>>(
        a.partial, plan.splits, items, I, amp);
    return cudaGetLastError();
}

}  // namespace xs
