// Phase records (Sec. 3.1 direct method with q on the reciprocal lattice):
// the device side of the record of one (frame, slot).
#pragma once

#include "xs_internal.h"

namespace xs {

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

// atom j of slot k: the coprime-stride order of runs of kPermRun
__device__ __forceinline__ int64_t slot_index(const PhaseSrc& ps, int64_t k) {
    return ps.opt.perm_mul == 1 ? k
                                : (int64_t)(((uint64_t)(k / kPermRun) * (uint64_t)ps.opt.perm_mul) %
                                            (uint64_t)(ps.n_pad / kPermRun)) * kPermRun + k % kPermRun;
}

// atom j of the call: its index in the positions and its form factor; false
// for padding slots
__device__ __forceinline__ bool atom_of(const PhaseSrc& ps, int64_t j, int64_t& a, float& fj, int* err) {
    if (!XS_IN_BOUNDS(err, j >= 0 && j < ps.n_pad)) return false;
    if (j >= ps.n_atoms) return false;
    // atom j of this call is atom a of the frames (a subset when an index is given)
    a = ps.opt.index ? (int64_t)ps.opt.index[j] : j;
    if (!XS_IN_BOUNDS(err, a >= 0 && a < (ps.opt.index ? ps.opt.pos_atoms : ps.n_atoms))) return false;
    fj = ps.f[a];
    return true;
}

__device__ __forceinline__ bool slot_atom(const PhaseSrc& ps, int64_t k, int64_t& a, float& fj, int* err) {
    return atom_of(ps, slot_index(ps, k), a, fj, err);
}

// position of atom a in frame t
__device__ __forceinline__ void pos_of(const PhaseSrc& ps, int64_t t, int64_t a, float& x, float& y, float& z) {
    const int64_t stride = ps.opt.index ? ps.opt.pos_atoms : ps.n_atoms;
    const int64_t idx = t * stride + a;
    const float* p = ps.pos + idx * 3;
    if (ps.opt.pos8) {
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
}

// the record of a position and form factor: turn counts of h^-1 r, exact
// integer arithmetic for an orthorhombic cell, FP64 otherwise; a non-finite
// form factor or position, or one more than 2^18 cells out, gives f = 0 and
// sets kDevErrNonFinite
__device__ __forceinline__ AtomRec rec_from(const PhaseSrc& ps, float x, float y, float z, float fj, int* err) {
    const PhaseOpts& opt = ps.opt;
    AtomRec r;
    r.ux = r.uy = r.uz = 0u;
    r.f = 0.0f;
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
        const Mat3& hs = ps.hs;
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
    return r;
}

// the record of atom a (form factor fj) in frame t
__device__ __forceinline__ AtomRec rec_of_atom(const PhaseSrc& ps, int64_t t, int64_t a, float fj, int* err) {
    float x, y, z;
    pos_of(ps, t, a, x, y, z);
    return rec_from(ps, x, y, z, fj, err);
}

}  // namespace xs
