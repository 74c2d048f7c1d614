// Phase records and the plain FP32 direct sum (Algorithm 1, Sec. 3.1).
//
// phase_kernel: one thread per (frame, atom slot).  s = h^-1 r is reduced
//   to its fractional part per axis and quantised to a 32-bit turn count: in
//   exact integer arithmetic for an orthorhombic cell, in FP64 otherwise.
//   Every later phase n_x*U_x + n_y*U_y + n_z*U_z is exact integer
//   arithmetic modulo one turn.  Slots may hold the atoms in
//   a coprime-stride order of runs of 8 (slot 8q + r holds atom
//   8 (q*a mod n_pad/8) + r): summing in that order turns the coherent partial
//   sums of an ordered crystal into random walks, while a run of 8 atoms (two
//   FCC cells) is too short to add up coherently.  Threads follow the slots:
//   the records are written coalesced and the positions gathered, a warp
//   reading four contiguous 96-byte runs (scattering 16-byte records from
//   coalesced reads measured 2.6x slower).
//
// direct_kernel: the plain reference-rate kernel.  A block owns 256*PX pixels
//   of one frame and a range of atoms; atom records are staged in shared
//   memory 256 at a time.  Each (atom, pixel) costs one exact integer phase,
//   one FP32 sincospi and a compensated (Kahan) FP32 update of Re and Im; the
//   compensated sums of each 256-atom tile are merged into FP64 accumulators.
//   Plain FP32 sums would drift by ~n*eps on coherent sums (q = 0, Bragg
//   peaks), where every term has the same sign and size.  Atom ranges ("splits") give enough blocks
//   for small grids; their FP64 partial amplitudes are added in a fixed order
//   by reduce_kernel, so results are deterministic.
#include <cmath>

#include "xs_internal.h"
#include "xs_phase.cuh"

namespace xs {

namespace {

constexpr int kDirectThreads = 256;
constexpr int kDirectPX = 4;     // pixels per thread
constexpr int kAtomTile = 256;   // atom records staged per shared-memory tile


constexpr int kPhaseFrames = 8;  // frames per block of the phase kernel

// grid: x = blocks of 256 slots, y = groups of kPhaseFrames frames; the atom of
// a slot (one 64-bit modulo) is computed once and reused for every frame
__global__ void __launch_bounds__(256) phase_kernel(PhaseSrc ps, int64_t n_frames, int* err) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= ps.n_pad) return;
    int64_t a = 0;
    float fj = 0.0f;
    const bool real = slot_atom(ps, k, a, fj, err);
    const int64_t t0 = (int64_t)blockIdx.y * kPhaseFrames;
    const int64_t t1 = min(n_frames, t0 + kPhaseFrames);
    for (int64_t t = t0; t < t1; ++t) {
        AtomRec r;
        r.ux = r.uy = r.uz = 0u;
        r.f = 0.0f;
        if (real) r = rec_of_atom(ps, t, a, fj, err);
        ps.rec[t * ps.n_pad + k] = r;
    }
}

__device__ __forceinline__ void pixel_miller(int64_t p, const GridDesc& g, uint32_t& nx, uint32_t& ny,
                                             uint32_t& nz) {
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int iz = (int)(p / plane);
    const int64_t rem = p - (int64_t)iz * plane;
    const int iy = (int)(rem / g.nx);
    const int ix = (int)(rem - (int64_t)iy * g.nx);
    nx = (uint32_t)(g.nx0 + ix);
    ny = (uint32_t)(g.ny0 + iy);
    nz = (uint32_t)(g.nz0 + iz);
}

// grid: x = pixel blocks, y = frame, z = atom split
__global__ void __launch_bounds__(kDirectThreads)
direct_kernel(const AtomRec* __restrict__ rec, int64_t n_pad, int64_t n_frames, GridDesc g,
              const int32_t* __restrict__ pts, int64_t atoms_per_split, double2* __restrict__ partial,
              float* __restrict__ I, float* __restrict__ amp) {
    __shared__ uint4 s_rec[kAtomTile];
    const int64_t P = g.pixels();  // with a point list: nx = the number of points
    const int t = blockIdx.y;
    const int split = blockIdx.z;
    const int64_t a0 = (int64_t)split * atoms_per_split;
    const int64_t a1 = min(n_pad, a0 + atoms_per_split);
    const uint4* frame_rec = reinterpret_cast<const uint4*>(rec + (int64_t)t * n_pad);

    uint32_t nx[kDirectPX], ny[kDirectPX], nz[kDirectPX];
    int64_t pix[kDirectPX];
#pragma unroll
    for (int i = 0; i < kDirectPX; ++i) {
        pix[i] = ((int64_t)blockIdx.x * kDirectPX + i) * kDirectThreads + threadIdx.x;
        const int64_t pc = pix[i] < P ? pix[i] : P - 1;
        if (pts) {
            nx[i] = (uint32_t)pts[3 * pc];
            ny[i] = (uint32_t)pts[3 * pc + 1];
            nz[i] = (uint32_t)pts[3 * pc + 2];
        } else {
            pixel_miller(pc, g, nx[i], ny[i], nz[i]);
        }
    }
    float re[kDirectPX], im[kDirectPX], cre[kDirectPX], cim[kDirectPX];
    double dre[kDirectPX], dim[kDirectPX];
#pragma unroll
    for (int i = 0; i < kDirectPX; ++i) {
        re[i] = im[i] = cre[i] = cim[i] = 0.0f;
        dre[i] = dim[i] = 0.0;
    }
    for (int64_t k0 = a0; k0 < a1; k0 += kAtomTile) {
        const int nk = (int)min((int64_t)kAtomTile, a1 - k0);
        __syncthreads();
        if (threadIdx.x < nk) s_rec[threadIdx.x] = frame_rec[k0 + threadIdx.x];
        __syncthreads();
        for (int k = 0; k < nk; ++k) {
            const uint4 a = s_rec[k];
            const float fj = __uint_as_float(a.w);
#pragma unroll
            for (int i = 0; i < kDirectPX; ++i) {
                const uint32_t ph = nx[i] * a.x + ny[i] * a.y + nz[i] * a.z;
                float c, s;
                phase_to_cs(ph, c, s);
                // Kahan: y = term - carried error; the rounding of re + y is
                // recovered exactly as (t - re) - y
                const float yr = fmaf(fj, c, -cre[i]);
                const float tr = re[i] + yr;
                cre[i] = (tr - re[i]) - yr;
                re[i] = tr;
                const float yi = fmaf(fj, s, -cim[i]);
                const float ti = im[i] + yi;
                cim[i] = (ti - im[i]) - yi;
                im[i] = ti;
            }
        }
#pragma unroll
        for (int i = 0; i < kDirectPX; ++i) {
            dre[i] += (double)re[i] - (double)cre[i];
            dim[i] += (double)im[i] - (double)cim[i];
            re[i] = im[i] = cre[i] = cim[i] = 0.0f;
        }
    }
#pragma unroll
    for (int i = 0; i < kDirectPX; ++i) {
        if (pix[i] >= P) continue;
        if (partial) {
            partial[((int64_t)split * n_frames + t) * P + pix[i]] = make_double2(dre[i], dim[i]);
        } else {
            const int64_t o = (int64_t)t * P + pix[i];
            I[o] = (float)(dre[i] * dre[i] + dim[i] * dim[i]);
            if (amp) {
                amp[2 * o] = (float)dre[i];
                amp[2 * o + 1] = (float)dim[i];
            }
        }
    }
}

__global__ void reduce_kernel(const double2* __restrict__ partial, int splits, int64_t n_items,
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

bool make_phase_src(const float* pos, const float* f, int64_t n_atoms, int64_t n_pad, const Mat3& hinv,
                    const PhaseOpts& opt, AtomRec* rec, PhaseSrc& ps) {
    // atom of slot k = kPermRun ((k / kPermRun) a mod n_pad / kPermRun) + k mod
    // kPermRun; the products stay below 2^64
    if (opt.perm_mul != 1 && (n_pad >= ((int64_t)1 << 32) || n_pad % kPermRun != 0)) return false;
    ps.pos = pos;
    ps.f = f;
    ps.n_atoms = n_atoms;
    ps.n_pad = n_pad;
    ps.rec = rec;
    for (int i = 0; i < 9; ++i) ps.hs.a[i] = hinv.a[i] * 4294967296.0;
    PhaseOpts& o = ps.opt;
    o = opt;
    o.pos8 = ((uintptr_t)pos & 7u) == 0;
    // orthorhombic cells: |x| < lim_x keeps |hs_xx x| below 2^50 (the FP32
    // bound is rounded down, so the check is conservative)
    for (int a = 0; a < 3; ++a) {
        const double d = std::fabs(ps.hs.a[4 * a]);
        o.lim[a] = d > 0.0 ? std::nextafter((float)(1125899906842624.0 / d), 0.0f) : 3.0e38f;
        // d = cm 2^ce with cm < 2^53 an integer (exact: frexp only moves the exponent)
        int e = 0;
        const double fr = std::frexp(d, &e);
        const uint64_t cm = (uint64_t)std::ldexp(fr, 53);
        o.ch[a] = (uint32_t)(cm >> 32);
        o.cl[a] = (uint32_t)cm;
        o.ce[a] = e - 53;
        o.cneg[a] = ps.hs.a[4 * a] < 0.0 ? 1u : 0u;
    }
    return true;
}

cudaError_t launch_phase(const float* pos, const float* f, int64_t n_atoms, int64_t n_frames,
                         int64_t n_pad, const Mat3& hinv, const PhaseOpts& opt, AtomRec* rec, int* err,
                         cudaStream_t st) {
    if (n_frames * n_pad == 0) return cudaSuccess;
    const int64_t gy = (n_frames + kPhaseFrames - 1) / kPhaseFrames;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    PhaseSrc ps;
    if (!make_phase_src(pos, f, n_atoms, n_pad, hinv, opt, rec, ps)) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((n_pad + 255) / 256), (unsigned)gy);
    ++tl_kernel_launches;
    phase_kernel<<<grid, 256, 0, st>>>(ps, n_frames, err);
    return cudaGetLastError();
}

DirectPlan plan_direct(int64_t n_pad, int64_t n_frames, const GridDesc& g, int num_sms) {
    DirectPlan p;
    const int64_t P = g.pixels();
    const int64_t pix_blocks = (P + kDirectThreads * kDirectPX - 1) / (kDirectThreads * kDirectPX);
    const int64_t base = pix_blocks * n_frames;
    const int64_t want = 2 * (int64_t)num_sms;
    int64_t tiles = (n_pad + kAtomTile - 1) / kAtomTile;
    int64_t splits = base >= want ? 1 : (want + base - 1) / base;
    if (splits > tiles) splits = tiles;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    const int64_t tiles_per = (tiles + splits - 1) / splits;
    p.atoms_per_split = tiles_per * kAtomTile;
    p.splits = (int)((tiles + tiles_per - 1) / tiles_per);
    if (p.splits < 1) p.splits = 1;
    p.partial_bytes = p.splits > 1 ? (size_t)p.splits * n_frames * P * sizeof(double2) : 0;
    return p;
}

cudaError_t launch_direct(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g,
                          const DirectPlan& plan, void* partial, float* I, float* amp,
                          cudaStream_t st, const int32_t* pts) {
    const int64_t P = g.pixels();
    if (P == 0 || n_frames == 0) return cudaSuccess;
    const int64_t pix_blocks = (P + kDirectThreads * kDirectPX - 1) / (kDirectThreads * kDirectPX);
    if (n_frames > 65535 || pix_blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)pix_blocks, (unsigned)n_frames, (unsigned)plan.splits);
    double2* part = plan.splits > 1 ? static_cast<double2*>(partial) : nullptr;
    ++tl_kernel_launches;
    direct_kernel<<<grid, kDirectThreads, 0, st>>>(rec, n_pad, n_frames, g, pts, plan.atoms_per_split, part, I,
                                                   amp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || plan.splits == 1) return e;
    const int64_t items = n_frames * P;
    const int64_t blocks = min((items + 255) / 256, (int64_t)65536);
    ++tl_kernel_launches;
    reduce_kernel<<<(unsigned)blocks, 256, 0, st>>>(part, plan.splits, items, I, amp);
    return cudaGetLastError();
}

}  // namespace xs
