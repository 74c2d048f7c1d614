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

namespace xs {

namespace {

constexpr int kDirectThreads = 256;
constexpr int kDirectPX = 4;     // pixels per thread
constexpr int kAtomTile = 256;   // atom records staged per shared-memory tile

// hs = 2^32 h^-1 (a power-of-two scaling, exact): rint(hs r) mod 2^32 equals
// rint(frac(h^-1 r) 2^32) mod 2^32.  Adding M = 1.5 * 2^52 to |v| < 2^51 gives
// M + rint(v) (ties to even) in one FP64 rounding, and the low 32 bits of that
// sum's encoding are rint(v) mod 2^32.
constexpr double kRoundMagic = 6755399441055744.0;      // 1.5 * 2^52
constexpr double kTurnLimit = 1125899906842624.0;       // 2^50: |v| bound checked
__device__ __forceinline__ uint32_t turns_of(double v) { return (uint32_t)__double2loint(v + kRoundMagic); }

// The count for an orthorhombic cell in integer arithmetic: x = +-m 2^ex
// (m the float's 24-bit significand) times c = +-cm 2^ce (cm < 2^53) is the
// exact product m cm = H 2^32 + L (two 32 x 32 -> 64-bit multiplies, H <
// 2^45) scaled by 2^-d, d = -(ex + ce).  The turns are bits d.. of m cm,
// rounded to nearest with ties to even from the bit below (rb) and those
// under it (sticky), as the FP64 rounding above does.  GB300 issues FP64 at a
// small fraction of its integer rate, and this was the phase kernel's only
// FP64 work.
__device__ __forceinline__ uint32_t turns_int(float x, uint32_t ch, uint32_t cl, int ce, uint32_t cneg) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t E = (b >> 23) & 0xffu;
    const uint32_t m = E ? ((b & 0x7fffffu) | 0x800000u) : (b & 0x7fffffu);
    const int d = -((E ? (int)E - 150 : -149) + ce);
    const uint64_t A = (uint64_t)m * cl;
    const uint64_t H = (uint64_t)m * ch + (A >> 32);
    const uint32_t L = (uint32_t)A;
    uint32_t u;
    if (d > 32 && d <= 77) {  // the usual case: |x c| < 2^45
        const int e = d - 32;
        const uint32_t q = (uint32_t)(H >> e);
        const uint32_t rb = (uint32_t)(H >> (e - 1)) & 1u;
        const uint32_t st = ((H & ((1ull << (e - 1)) - 1ull)) != 0ull || L != 0u) ? 1u : 0u;
        u = q + (rb & (st | (q & 1u)));
    } else if (d > 77) {
        u = 0u;  // |x c| < 1/2
    } else if (d > 0) {
        const uint32_t q = d == 32 ? (uint32_t)H : (((uint32_t)H << (32 - d)) | (L >> d));
        const uint32_t rb = (L >> (d - 1)) & 1u;
        const uint32_t st = (L & ((1u << (d - 1)) - 1u)) != 0u ? 1u : 0u;
        u = q + (rb & (st | (q & 1u)));
    } else {
        u = d <= -32 ? 0u : L << -d;
    }
    return ((b >> 31) ^ cneg) ? 0u - u : u;
}

constexpr int kPhaseFrames = 8;  // frames per block of the phase kernel

// grid: x = blocks of 256 slots, y = groups of kPhaseFrames frames; the atom of
// a slot (one 64-bit modulo) is computed once and reused for every frame
__global__ void __launch_bounds__(256)
phase_kernel(const float* __restrict__ pos, const float* __restrict__ f, int64_t n_atoms, int64_t n_frames,
             int64_t n_pad, Mat3 hs, PhaseOpts opt, AtomRec* __restrict__ rec, int* err) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_pad) return;
    const int64_t j = opt.perm_mul == 1 ? k
                                        : (int64_t)(((uint64_t)(k / kPermRun) * (uint64_t)opt.perm_mul) %
                                                    (uint64_t)(n_pad / kPermRun)) * kPermRun + k % kPermRun;
    if (!XS_IN_BOUNDS(err, j >= 0 && j < n_pad)) return;
    const bool real = j < n_atoms;
    // atom j of this call is atom a of the frames (a subset when an index is given)
    const int64_t a = (opt.index && real) ? (int64_t)opt.index[j] : j;
    const int64_t stride = opt.index ? opt.pos_atoms : n_atoms;
    if (real && !XS_IN_BOUNDS(err, a >= 0 && a < stride)) return;
    const float fj = real ? f[a] : 0.0f;
    const int64_t t0 = (int64_t)blockIdx.y * kPhaseFrames;
    const int64_t t1 = min(n_frames, t0 + kPhaseFrames);
    for (int64_t t = t0; t < t1; ++t) {
        AtomRec r;
        r.ux = r.uy = r.uz = 0u;
        r.f = 0.0f;
        if (real) {
            const int64_t idx = t * stride + a;
            const float* p = pos + idx * 3;
            float x, y, z;
            if (opt.pos8) {
                // with `pos` 8-byte aligned, the 12-byte position is one aligned
                // 8-byte load and one 4-byte load: (x, y) + z at an even index,
                // x + (y, z) at an odd one
                const int odd = (int)(idx & 1);
                const float2 v2 = *reinterpret_cast<const float2*>(p + odd);
                const float v1 = p[odd ? 0 : 2];
                x = odd ? v1 : v2.x;
                y = odd ? v2.x : v2.y;
                z = odd ? v2.y : v1;
            } else {
                x = p[0];
                y = p[1];
                z = p[2];
            }
            // NaN and Inf fail these comparisons too
            bool ok = isfinite(fj);
            if (opt.ortho) {
                ok = ok && fabsf(x) < opt.lim[0] && fabsf(y) < opt.lim[1] && fabsf(z) < opt.lim[2];
                if (ok) {
                    r.ux = turns_int(x, opt.ch[0], opt.cl[0], opt.ce[0], opt.cneg[0]);
                    r.uy = turns_int(y, opt.ch[1], opt.cl[1], opt.ce[1], opt.cneg[1]);
                    if (opt.need_z) r.uz = turns_int(z, opt.ch[2], opt.cl[2], opt.ce[2], opt.cneg[2]);
                }
            } else {
                const double vx = hs.a[0] * x + hs.a[1] * y + hs.a[2] * z;
                const double vy = hs.a[3] * x + hs.a[4] * y + hs.a[5] * z;
                const double vz = hs.a[6] * x + hs.a[7] * y + hs.a[8] * z;
                ok = ok && fabs(vx) < kTurnLimit && fabs(vy) < kTurnLimit && fabs(vz) < kTurnLimit;
                if (ok) {
                    r.ux = turns_of(vx);
                    r.uy = turns_of(vy);
                    if (opt.need_z) r.uz = turns_of(vz);
                }
            }
            if (ok)
                r.f = fj;
            else
                set_dev_error(err, kDevErrNonFinite);
        }
        rec[t * n_pad + k] = r;
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

cudaError_t launch_phase(const float* pos, const float* f, int64_t n_atoms, int64_t n_frames,
                         int64_t n_pad, const Mat3& hinv, const PhaseOpts& opt, AtomRec* rec, int* err,
                         cudaStream_t st) {
    if (n_frames * n_pad == 0) return cudaSuccess;
    const int64_t gy = (n_frames + kPhaseFrames - 1) / kPhaseFrames;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    Mat3 hs;
    for (int i = 0; i < 9; ++i) hs.a[i] = hinv.a[i] * 4294967296.0;
    PhaseOpts o = opt;
    o.pos8 = ((uintptr_t)pos & 7u) == 0;
    // atom of slot k = kPermRun ((k / kPermRun) a mod n_pad / kPermRun) + k mod
    // kPermRun; the products stay below 2^64
    if (o.perm_mul != 1 && (n_pad >= ((int64_t)1 << 32) || n_pad % kPermRun != 0)) return cudaErrorInvalidValue;
    // orthorhombic cells: |x| < lim_x keeps |hs_xx x| below 2^50 (the FP32
    // bound is rounded down, so the check is conservative)
    for (int a = 0; a < 3; ++a) {
        const double d = std::fabs(hs.a[4 * a]);
        o.lim[a] = d > 0.0 ? std::nextafter((float)(1125899906842624.0 / d), 0.0f) : 3.0e38f;
        // d = cm 2^ce with cm < 2^53 an integer (exact: frexp only moves the exponent)
        int e = 0;
        const double fr = std::frexp(d, &e);
        const uint64_t cm = (uint64_t)std::ldexp(fr, 53);
        o.ch[a] = (uint32_t)(cm >> 32);
        o.cl[a] = (uint32_t)cm;
        o.ce[a] = e - 53;
        o.cneg[a] = hs.a[4 * a] < 0.0 ? 1u : 0u;
    }
    dim3 grid((unsigned)((n_pad + 255) / 256), (unsigned)gy);
    ++tl_kernel_launches;
    phase_kernel<<<grid, 256, 0, st>>>(pos, f, n_atoms, n_frames, n_pad, hs, o, rec, err);
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
