// Tensor-core kernels of the adjoint (k_adjoint.cu forms H and launches them).
//
// With H_q = G_q conj(S_q) and rows q = (n_x, n_z) of the grid,
//   Z(q, j)   = sum_y H(q, y) E_y(y, j),    Z_y(q, j) = sum_y n_y H(q, y) E_y(y, j),
// E_y(y, j) = exp(i 2 pi n_y U_y(j) / 2^32), is a complex matrix product with
// K = n_y, and the gradient needs per atom
//   Im T_x = sum_q n_x Im[E_xz Z],  Im T_y = sum_q Im[E_xz Z_y],  Im T_z = sum_q n_z Im[E_xz Z],
// E_xz(q, j) = exp(i 2 pi (n_x U_x(j) + n_z U_z(j)) / 2^32) (Sec. 3.1 factorisation).
//
// The complex product is a real one with the real and imaginary parts folded
// into K: k' = 2 y + p, and per complex row q four real rows
//   [Re H, -Im H] -> Re Z      [Im H, Re H] -> Im Z
//   n_y [Re H, -Im H] -> Re Z_y  n_y [Im H, Re H] -> Im Z_y
// against B[j][2y + p] = (Re E_y, Im E_y), so every accumulator element is a
// finished real or imaginary part.  In a row tile, rows 2q' + p' (p' = 0, 1:
// real, imaginary part) of the first 64 hold Z and those of the last 64 hold
// Z_y, so each warp holds one kind.  adjoint_image_kernel writes A as split
// BF16 (hi + lo; H exceeds the FP16 range) already in the shared-memory
// layout the tensor core reads (MN-major, 128-byte swizzle), one 16 KB image
// per (row tile of 32 q, stage of 16 n_y).
//
// adjoint_tc_kernel: one CTA of 128 threads owns 128 atoms.  Per row tile and
// stage it copies the A image, builds B (one thread per atom, exact integer
// phases) and one thread issues 2 K-steps x 3 split passes of
// tcgen05.mma.cta_group::1 (M = N = 128) into 128 TMEM columns; then each
// thread owns one accumulator row: it forms E_xz times its part of Z or Z_y,
// the row sums go over lanes by a transposed butterfly (lane l ends with
// atom column l of 32) and over warps in a fixed order, and each thread keeps
// the running Im T of its atom.  Two 32 KB stage buffers: one is filled while
// the other is multiplied; three CTAs share an SM.  Every wait is bounded.
#include <cuda_bf16.h>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kAtAtoms = 128;                       // MMA N: atoms per CTA
constexpr int kAtRows = 128;                        // MMA M: 32 complex rows x 4
constexpr int kAtQ = kAtRows / 4;                   // complex rows per row tile
constexpr int kAtK = 32;                            // k' per stage (16 n_y)
constexpr int kAtThreads = 128;
constexpr uint32_t kAtBlock = (kAtK / 8) * 1024;    // 64-row MN block: 4 KB
constexpr uint32_t kAtHalf = 2 * kAtBlock;          // 128 rows of one operand half
constexpr uint32_t kAtImage = 2 * kAtHalf;          // A hi + lo of one (row tile, stage)
constexpr uint32_t kAtStage = 4 * kAtHalf;          // A hi, A lo, B hi, B lo: 32 KB
constexpr int kAtBufs = 2;                          // stage buffers: fill one while the other multiplies
constexpr int kAtTab = 256;

struct AtCtl {
    uint64_t done[kAtBufs];
    uint64_t drain;
    uint32_t tmem;
    int abort;
    float2 tab[kAtTab];      // exp(i 2 pi k / 256)
    AtomRec rec[kAtAtoms];
};
// the warps' row sums [warp][atom][2 of 3] reuse the stage buffers: warps 0-1
// the n_x- and n_z-weighted sums of Im[E Z], warps 2-3 the sum of Im[E Z_y]
static_assert(4 * kAtAtoms * 3 * sizeof(float) <= kAtBufs * kAtStage, "row sums fit in the stage buffers");

constexpr size_t kAtSmemBytes = 1024 + kAtBufs * kAtStage + sizeof(AtCtl);

// byte offset of the 16-byte chunk holding MN rows [mn, mn+8) of K row k
__host__ __device__ __forceinline__ uint32_t at_chunk(int mn, int k) {
    return (uint32_t)(mn >> 6) * kAtBlock + (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * 128u +
           ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4);
}

__device__ __forceinline__ uint32_t at_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void at_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(at_smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool at_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(at_smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// bounded wait; false if aborted or timed out (which also raises the abort flag)
__device__ bool at_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int64_t timeout_ns) {
    if (at_try_wait(bar, parity, 0u)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (at_try_wait(bar, parity, 20000u)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(globaltimer_ns() - t0) > timeout_ns) {
            *abort_flag = 1;
            set_dev_error(err, kDevErrTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void at_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void at_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// MN-major, 128-byte swizzle: leading byte offset = stride between 64-row MN
// blocks, stride byte offset = stride between 8-row K atoms
__device__ __forceinline__ uint64_t at_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kAtBlock >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// kind::f16 instruction descriptor: FP32 D, BF16 A and B, both MN-major, M, N
__host__ __device__ constexpr uint32_t at_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void at_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void at_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     at_smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void at_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void at_wait_ld(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// exp(i 2 pi P / 2^32): table value of the top 8 bits times Taylor polynomials
// of the remaining angle t < 2 pi / 256 (truncation below 3e-13)
__device__ __forceinline__ float2 at_cis(uint32_t P, const float2* tab) {
    const float2 a = tab[P >> 24];
    const float t = (float)(P & 0xFFFFFFu) * 1.4629180792671596e-9f;  // 2 pi / 2^32
    const float t2 = t * t;
    const float c = fmaf(t2, fmaf(t2, 1.0f / 24.0f, -0.5f), 1.0f);
    const float s = t * fmaf(t2, fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

__device__ __forceinline__ void at_split(float v, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// one thread per element (row tile, stage, row m, k') of the A images
__global__ void adjoint_image_kernel(const float2* __restrict__ H, GridDesc g, int n_mtiles, int n_stages,
                                     uint8_t* __restrict__ img) {
    const int64_t n = (int64_t)n_mtiles * n_stages * kAtRows * kAtK;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int kk = (int)(i % kAtK);
    const int m = (int)((i / kAtK) % kAtRows);
    const int64_t ts = i / ((int64_t)kAtK * kAtRows);  // mt * n_stages + s
    const int s = (int)(ts % n_stages);
    const int64_t mt = ts / n_stages;
    const int64_t q = mt * kAtQ + ((m & 63) >> 1);
    const bool im_row = (m & 1) != 0;
    const bool zy_row = m >= 64;
    const int y = s * (kAtK / 2) + (kk >> 1);
    const int p = kk & 1;
    float v = 0.0f;
    if (q < (int64_t)g.nx * g.nz && y < g.ny) {
        const int64_t x = q % g.nx, z = q / g.nx;
        const float2 h = H[(z * g.ny + y) * g.nx + x];
        v = p == 0 ? (im_row ? h.y : h.x) : (im_row ? h.x : -h.y);
        if (zy_row) v *= (float)(g.ny0 + y);
    }
    uint16_t hi, lo;
    at_split(v, hi, lo);
    uint8_t* base = img + ts * kAtImage + at_chunk(m, kk) + (uint32_t)(m & 7) * 2u;
    *reinterpret_cast<uint16_t*>(base) = hi;
    *reinterpret_cast<uint16_t*>(base + kAtHalf) = lo;
}

__global__ void __launch_bounds__(kAtThreads)
adjoint_tc_kernel(const AtomRec* __restrict__ rec, int64_t n_atoms, int64_t n_pad, GridDesc g, Mat3 hinv,
                  const uint8_t* __restrict__ img, int n_mtiles, int n_stages, float* __restrict__ grad, int* err,
                  int64_t timeout_ns) {
    extern __shared__ __align__(16) uint8_t at_raw[];
    const uint32_t raw = at_smem_u32(at_raw);
    uint8_t* smem = at_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t stage = at_smem_u32(smem);
    AtCtl* ctl = reinterpret_cast<AtCtl*>(smem + kAtBufs * kAtStage);
    float* red = reinterpret_cast<float*>(smem);  // [warp][atom][3], between stages
    volatile int* abort_flag = &ctl->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile0 = (int64_t)blockIdx.x * kAtAtoms;

    for (int i = tid; i < kAtTab; i += kAtThreads) {
        double s, c;
        sincospi((double)i / (kAtTab / 2), &s, &c);
        ctl->tab[i] = make_float2((float)c, (float)s);
    }
    {
        AtomRec a;
        a.ux = a.uy = a.uz = 0u;
        a.f = 0.0f;
        if (tile0 + tid < n_pad) a = rec[tile0 + tid];  // the last tile may reach past n_pad
        ctl->rec[tid] = a;
    }
    if (tid == 0) {
        for (int b = 0; b < kAtBufs; ++b) at_mbar_init(&ctl->done[b], 1);
        at_mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         at_smem_u32(&ctl->tmem)),
                     "r"((uint32_t)kAtAtoms)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    at_fence_before();
    __syncthreads();
    at_fence_after();
    const uint32_t tmem = ctl->tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    constexpr uint32_t idesc = at_idesc(kAtRows, kAtAtoms);
    const AtomRec me = ctl->rec[tid];
    const int64_t Q = (int64_t)g.nx * g.nz;
    // this thread's B row (MN = tid): block, byte in the chunk, and the swizzled
    // chunk of each of the 8 K rows of an atom
    const uint32_t b_row = (uint32_t)(tid >> 6) * kAtBlock + (uint32_t)(tid & 7) * 2u;
    uint32_t b_off[8];
#pragma unroll
    for (int kr = 0; kr < 8; ++kr) b_off[kr] = (uint32_t)kr * 128u + ((uint32_t)(((tid & 63) >> 3) ^ kr) << 4);
    const float2 w_step = at_cis(me.uy, ctl->tab);

    float tx = 0.0f, ty = 0.0f, tz = 0.0f;  // Im T of this thread's atom
    // each commit completes one phase of its buffer's barrier; every phase is
    // waited for exactly once: before the buffer is filled again, or at the end
    // of a row tile (older buffer first)
    uint32_t phases = 0u, pend = 0u;  // bit b: buffer b's barrier parity, commit not yet waited for
    int64_t issued = 0;
    bool ok = true;
    for (int mt = 0; mt < n_mtiles && ok; ++mt) {
        for (int s = 0; s < n_stages && ok; ++s) {
            const int bs = (int)(issued & 1);
            if ((pend >> bs) & 1u) {
                ok = at_wait(&ctl->done[bs], (phases >> bs) & 1u, abort_flag, err, timeout_ns);
                phases ^= 1u << bs;
                pend &= ~(1u << bs);
                if (!ok) break;
                at_fence_after();
            }
            uint8_t* buf = smem + (uint32_t)bs * kAtStage;
            const uint32_t bufa = stage + (uint32_t)bs * kAtStage;
            // A: copy the image of (mt, s); B: E_y of this thread's atom, from an
            // exact seed per stage and the exact step exp(i 2 pi U_y) (16 FP32
            // rotations stay far below the split format's resolution)
            const uint4* src = reinterpret_cast<const uint4*>(img + ((int64_t)mt * n_stages + s) * kAtImage);
            uint4* dst = reinterpret_cast<uint4*>(buf);
            uint4 tmp[kAtImage / 16 / kAtThreads];
#pragma unroll
            for (int i = 0; i < (int)(kAtImage / 16 / kAtThreads); ++i) tmp[i] = src[i * kAtThreads + tid];
#pragma unroll
            for (int i = 0; i < (int)(kAtImage / 16 / kAtThreads); ++i) dst[i * kAtThreads + tid] = tmp[i];
            const int y0 = s * (kAtK / 2);
            float2 e = at_cis((uint32_t)(g.ny0 + y0) * me.uy, ctl->tab);
#pragma unroll
            for (int yy = 0; yy < kAtK / 2; ++yy) {
                const float2 ev = (y0 + yy < g.ny) ? e : make_float2(0.0f, 0.0f);
                uint16_t h0, l0, h1, l1;
                at_split(ev.x, h0, l0);
                at_split(ev.y, h1, l1);
                // k' = 2 yy and 2 yy + 1: K atom yy / 4, rows (2 yy) & 7 and (2 yy + 1) & 7
                uint8_t* r0 = buf + b_row + (uint32_t)(yy >> 2) * 1024u + b_off[(2 * yy) & 7];
                uint8_t* r1 = buf + b_row + (uint32_t)(yy >> 2) * 1024u + b_off[(2 * yy + 1) & 7];
                *reinterpret_cast<uint16_t*>(r0 + 2 * kAtHalf) = h0;
                *reinterpret_cast<uint16_t*>(r0 + 3 * kAtHalf) = l0;
                *reinterpret_cast<uint16_t*>(r1 + 2 * kAtHalf) = h1;
                *reinterpret_cast<uint16_t*>(r1 + 3 * kAtHalf) = l1;
                e = make_float2(fmaf(e.x, w_step.x, -e.y * w_step.y), fmaf(e.x, w_step.y, e.y * w_step.x));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                at_fence_after();
                const uint32_t a_hi = bufa, a_lo = bufa + kAtHalf, b_hi = bufa + 2 * kAtHalf, b_lo = bufa + 3 * kAtHalf;
#pragma unroll
                for (int kk = 0; kk < kAtK / 16; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 2048u;  // two 8-row K atoms per K = 16
                    at_mma(tmem, at_desc(a_hi + ko), at_desc(b_hi + ko), idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    at_mma(tmem, at_desc(a_hi + ko), at_desc(b_lo + ko), idesc, 1u);
                    at_mma(tmem, at_desc(a_lo + ko), at_desc(b_hi + ko), idesc, 1u);
                }
                at_commit(&ctl->done[bs]);
            }
            pend |= 1u << bs;
            ++issued;
        }
        if (!ok) break;
        // the row tile's last MMAs: then both buffers are free and the
        // accumulator final
        for (int k = 0; k < kAtBufs && ok; ++k) {
            const int bb = (int)((issued + k) & 1);
            if ((pend >> bb) & 1u) {
                ok = at_wait(&ctl->done[bb], (phases >> bb) & 1u, abort_flag, err, timeout_ns);
                phases ^= 1u << bb;
                pend &= ~(1u << bb);
            }
        }
        if (!ok) break;
        at_fence_after();
        // epilogue: this thread's accumulator row m = tid; warps 0-1 hold Z,
        // warps 2-3 hold Z_y; even rows real parts, odd rows imaginary parts
        const int64_t q = (int64_t)mt * kAtQ + ((tid & 63) >> 1);
        const bool im_row = (tid & 1) != 0;
        const bool z_warp = warp < 2;
        int nxv = 0, nzv = 0;
        if (q < Q) {
            nxv = g.nx0 + (int)(q % g.nx);
            nzv = g.nz0 + (int)(q / g.nx);
        }
        const float wa = (q < Q) ? (z_warp ? (float)nxv : 1.0f) : 0.0f;
        const float wb = (q < Q) ? (float)nzv : 0.0f;
        for (int c32 = 0; c32 < kAtAtoms / 32; ++c32) {
            uint32_t v[32];
            at_ld16(lane_base + (uint32_t)(c32 * 32), v);
            at_ld16(lane_base + (uint32_t)(c32 * 32 + 16), v + 16);
            at_wait_ld(v);
            at_wait_ld(v + 16);
            // Im[E X] = Re E Im X + Im E Re X, weighted by n_x (or 1) and n_z
            float a[32], b[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const AtomRec& aj = ctl->rec[c32 * 32 + k];
                const float2 e = at_cis((uint32_t)nxv * aj.ux + (uint32_t)nzv * aj.uz, ctl->tab);
                const float c = (im_row ? e.x : e.y) * __uint_as_float(v[k]);
                a[k] = wa * c;
                b[k] = wb * c;
            }
            // transposed butterfly: at offset o the lanes with bit o keep the
            // upper half of their values; lane l ends with the sum of column l
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int k = 0; k < o; ++k) {
                    const float sa = up ? a[k] : a[k + o];
                    a[k] = (up ? a[k + o] : a[k]) + __shfl_xor_sync(0xffffffffu, sa, o);
                    if (z_warp) {
                        const float sb = up ? b[k] : b[k + o];
                        b[k] = (up ? b[k + o] : b[k]) + __shfl_xor_sync(0xffffffffu, sb, o);
                    }
                }
            }
            float* rw = red + (warp * kAtAtoms + c32 * 32 + lane) * 3;
            rw[0] = a[0];
            rw[1] = b[0];
        }
        at_fence_before();
        __syncthreads();
        // warps 0-1: (n_x-weighted, n_z-weighted) sums of Im[E Z]; warps 2-3: Im[E Z_y]
        tx += red[(0 * kAtAtoms + tid) * 3 + 0] + red[(1 * kAtAtoms + tid) * 3 + 0];
        tz += red[(0 * kAtAtoms + tid) * 3 + 1] + red[(1 * kAtAtoms + tid) * 3 + 1];
        ty += red[(2 * kAtAtoms + tid) * 3 + 0] + red[(3 * kAtAtoms + tid) * 3 + 0];
        __syncthreads();
        at_fence_after();
    }
    if (ok) {
        const int64_t j = tile0 + tid;
        if (j < n_atoms) {
            const double scale = -4.0 * 3.14159265358979323846 * (double)me.f;
            const double v[3] = {(double)tx, (double)ty, (double)tz};
            for (int c = 0; c < 3; ++c) {
                const double hv = hinv.a[0 * 3 + c] * v[0] + hinv.a[1 * 3 + c] * v[1] + hinv.a[2 * 3 + c] * v[2];
                grad[j * 3 + c] = (float)(scale * hv);
            }
        }
    } else if (tid == 0) {
        // every issued MMA must finish before tensor memory is released
        at_commit(&ctl->drain);
        int no_abort = 0;
        at_wait(&ctl->drain, 0u, &no_abort, err, 2000000000LL);
    }
    at_fence_before();
    __syncthreads();
    if (warp == 0) {
        at_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kAtAtoms)
                     : "memory");
    }
}

}  // namespace

size_t adjoint_tc_image_bytes(const GridDesc& g) {
    const int64_t n_mtiles = ((int64_t)g.nx * g.nz + kAtQ - 1) / kAtQ;
    const int64_t n_stages = ((int64_t)g.ny + kAtK / 2 - 1) / (kAtK / 2);
    return (size_t)(n_mtiles * n_stages) * kAtImage;
}

cudaError_t launch_adjoint_tc(const AtomRec* rec, int64_t n_atoms, int64_t n_pad, const GridDesc& g,
                              const Mat3& hinv, const float2* H, void* image, float* grad, int* err,
                              int64_t timeout_ns, cudaStream_t st) {
    const int64_t n_mtiles = ((int64_t)g.nx * g.nz + kAtQ - 1) / kAtQ;
    const int64_t n_stages = ((int64_t)g.ny + kAtK / 2 - 1) / (kAtK / 2);
    if (n_mtiles > INT32_MAX || n_stages > INT32_MAX) return cudaErrorInvalidValue;
    uint8_t* img = static_cast<uint8_t*>(image);
    const int64_t n_el = n_mtiles * n_stages * kAtRows * kAtK;
    ++tl_kernel_launches;
    adjoint_image_kernel<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(H, g, (int)n_mtiles, (int)n_stages, img);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(adjoint_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAtSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (n_pad + kAtAtoms - 1) / kAtAtoms;
    ++tl_kernel_launches;
    adjoint_tc_kernel<<<(unsigned)blocks, kAtThreads, kAtSmemBytes, st>>>(rec, n_atoms, n_pad, g, hinv, img,
                                                                          (int)n_mtiles, (int)n_stages, grad, err,
                                                                          timeout_ns);
    return cudaGetLastError();
}

}  // namespace xs
