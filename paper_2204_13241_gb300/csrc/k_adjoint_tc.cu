// Tensor-core kernels of the adjoint (the sums they compute are derived in k_adjoint.cu).
//
// With H_q = G_q conj(S_q) and rows q = (n_x, n_z) of the grid,
//   Z(q, j)   = sum_y H(q, y) E_y(y, j),    Z_y(q, j) = sum_y n_y H(q, y) E_y(y, j),
// E_y(y, j) = exp(i 2 pi n_y U_y(j) / 2^32), is a complex matrix product with
// K = n_y, and the gradient needs per atom
//   Im T_x = sum_q n_x Im[E_xz Z],  Im T_y = sum_q Im[E_xz Z_y],  Im T_z = sum_q n_z Im[E_xz Z],
// E_xz(q, j) = exp(i 2 pi (n_x U_x(j) + n_z U_z(j)) / 2^32) (Sec. 3.1 factorisation).
//
// The complex product is a real one with the real and imaginary parts folded
// into K: k' = 2 y + p, and per complex row q four real rows ("kinds")
//   [Re H, -Im H] -> Re Z      [Im H, Re H] -> Im Z
//   n_y [Re H, -Im H] -> Re Z_y  n_y [Im H, Re H] -> Im Z_y
// against A[j][2y + p] = (Re E_y, Im E_y), so every accumulator element is a
// finished real or imaginary part.
//
// adjoint_tc_kernel: a pair of CTAs (cta_group::2) owns 256 atoms, 128 per
// CTA, which are the MMA's M rows; the N = 256 columns are one row tile of
// the H image: 64 complex rows q times the four kinds, Re Z and Im Z in CTA
// 0's half of B, Re Z_y and Im Z_y in CTA 1's.  Per stage (32 n_y, K' = 64):
//   * 8 producer warps per CTA write E_y of their CTA's 128 atoms in split
//     BF16 (hi + lo) into the K-major, 128-byte-swizzled layout, two threads
//     per atom and 16 n_y each, from a seed exp(i 2 pi n_y0 U_y) and the step
//     exp(i 2 pi U_y), as 16-byte chunks;
//   * one loader thread per CTA moves its half of the prebuilt H image
//     (hi + lo, MN-major, 128-byte swizzle, 32 KB) with one cp.async.bulk
//     from the workspace, completing on a barrier of its own;
//   * in CTA 1 a relay thread forwards the filled stage (producers and copy)
//     to CTA 0 with one cluster-scope release;
//   * one thread of CTA 0 issues 4 K-steps x 3 split passes (hi hi, hi lo,
//     lo hi) of tcgen05.mma (M = N = 256) into one of two TMEM accumulators;
//   * after a row tile, 4 epilogue warps per CTA read their atom's 256
//     columns (one TMEM lane = one atom), form Im[E_xz X] with E_xz advanced
//     along n_x by the exact step exp(i 2 pi U_x) (reseeded every 16 rows and
//     where n_x wraps) and write the atom's sums of the row tile, while the
//     MMA fills the other accumulator.
// Pairs are persistent over the units (tile of 256 atoms, row tile), dealt
// round-robin: cutting the work at row tiles instead of whole atom tiles
// shortens the last wave; adjoint_finish_kernel adds each atom's row-tile
// sums in row-tile order and forms the gradient.  Every wait is bounded; on
// expiry the kernel sets the device error word, all roles leave, the loader
// waits for its copies in flight and tensor memory is released.
#include <cuda_bf16.h>

#include <algorithm>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kAtAtomsCta = 128;                    // M rows per CTA (atoms)
constexpr int kAtN = 256;                           // MMA N: one row tile of the H image
constexpr int kAtQ = kAtN / 4;                      // complex rows q per row tile
constexpr int kAtK = 64;                            // k' per stage (32 n_y)
constexpr int kAtStages = 3;
constexpr int kAtProdWarps = 8;
constexpr int kAtEpiWarps = 4;
constexpr int kAtMmaWarp = 0, kAtLoadWarp = 1, kAtProdWarp0 = 6;  // warps 2-5: epilogue
constexpr int kAtThreads = (kAtProdWarp0 + kAtProdWarps) * 32;  // 448
constexpr uint32_t kAtAHalf = kAtAtomsCta * 128;    // K-major: 128 rows x 128 B (64 BF16 of K)
constexpr uint32_t kAtBBlock = (kAtK / 8) * 1024;   // MN-major: 64-row MN block of 8 K atoms, 8 KB
constexpr uint32_t kAtBHalf = 2 * kAtBBlock;        // 128 H rows of one CTA
constexpr uint32_t kAtBBytes = 2 * kAtBHalf;        // hi + lo: one bulk copy, 32 KB
constexpr uint32_t kAtStage = 2 * kAtAHalf + kAtBBytes;  // A hi, A lo, B hi, B lo: 64 KB
constexpr uint32_t kAtTmemCols = 512;               // two 256-column FP32 accumulators
constexpr int kAtTab = 256;

struct AtCtl {
    uint64_t full[kAtStages];   // CTA 0: its producer warps and the peer's relay
    uint64_t fill[kAtStages];   // CTA 1: its producer warps (forwarded by the relay)
    uint64_t copy[kAtStages];   // each CTA: its loader's bulk copy (transaction bytes)
    uint64_t empty[kAtStages];  // each CTA: MMA commits
    uint64_t acc_full[2];       // each CTA: MMA commits
    uint64_t acc_empty[2];      // CTA 0: epilogue warps of both CTAs
    uint64_t drain;
    uint32_t tmem;
    int abort;
    float2 tab[kAtTab];         // exp(i 2 pi k / 256)
};

constexpr size_t kAtSmemBytes = 1024 + kAtStages * (size_t)kAtStage + sizeof(AtCtl);

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ uint32_t at_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t at_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void at_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t at_map(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void at_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(at_smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void at_arrive_local(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(at_smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void at_arrive_cluster(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

__device__ __forceinline__ void at_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(at_smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> this CTA's shared memory, completing `bytes` on `bar`; addresses
// 16-byte aligned, size a multiple of 16
__device__ __forceinline__ void at_bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"((uint64_t)__cvta_generic_to_global(src)), "r"(bytes), "r"(at_smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool at_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(at_smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// bounded wait; false if aborted or timed out (which also raises the abort flag)
__device__ bool at_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int64_t timeout_ns,
                        uint32_t hint_ns = 20000u) {
    if (at_try_wait(bar, parity, 0u)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (at_try_wait(bar, parity, hint_ns)) return true;
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

// B (H image): MN-major, 128-byte swizzle; leading byte offset = stride
// between 64-row MN blocks, stride byte offset = stride between 8-row K atoms
__device__ __forceinline__ uint64_t at_desc_mn(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kAtBBlock >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// A (E_y): K-major, 128-byte swizzle: rows of 128 B (64 BF16 of K), stride
// byte offset = stride between 8-row groups (1024 B); the leading byte offset
// is not used by swizzled K-major layouts.  A K step of 16 advances the start
// address by 32 B inside the swizzle row.
__device__ __forceinline__ uint64_t at_desc_k(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// kind::f16 instruction descriptor: FP32 D, BF16 A (K-major) and B (MN-major)
__host__ __device__ constexpr uint32_t at_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void at_mma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on `bar` in the CTAs of `mask` once every tcgen05 operation issued so
// far by this thread completes
__device__ __forceinline__ void at_commit_pair(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            at_smem_u32(bar)),
        "h"(mask)
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

__device__ __forceinline__ void at_st_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
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

__device__ __forceinline__ float2 at_cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// (re, im) -> packed BF16 hi = (RN(re), RN(im)) and lo = (RN(re - hi), RN(im - hi))
__device__ __forceinline__ void at_split2(float2 v, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    const float2 hv = __bfloat1622float2(h);
    const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(v.x - hv.x, v.y - hv.y));
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void at_split(float v, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// byte offset of the 16-byte chunk holding MN rows [mn, mn+8) of K row k in
// an MN-major, 128-byte-swizzled half of 2 MN blocks
__host__ __device__ __forceinline__ uint32_t at_chunk_mn(int mn, int k) {
    return (uint32_t)(mn >> 6) * kAtBBlock + (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * 128u +
           ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4);
}

// The H image: per (row tile rt, stage s, CTA half r) 32 KB = [hi 16 KB | lo
// 16 KB] of 128 rows (kind 2r + (row >> 6), q = 64 rt + (row & 63)) by 64 k'
// (n_y = 32 s + k' / 2), MN-major with 128-byte swizzle.  One thread per
// element (hi and lo), which forms H_q = G_q conj(S_q) from the amplitude
// (interleaved re, im) and dL/dI where it reads them.
__global__ void adjoint_image_kernel(const float* __restrict__ amp, const float* __restrict__ G, GridDesc g,
                                     int n_rt, int n_st, uint8_t* __restrict__ img) {
    const int64_t n = (int64_t)n_rt * n_st * 2 * 128 * kAtK;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int kk = (int)(i % kAtK);
    const int row = (int)((i / kAtK) % 128);
    const int64_t blk = i / ((int64_t)kAtK * 128);  // (rt n_st + s) 2 + r
    const int r = (int)(blk & 1);
    const int64_t ts = blk >> 1;
    const int s = (int)(ts % n_st);
    const int64_t rt = ts / n_st;
    const int kind = 2 * r + (row >> 6);
    const int64_t q = rt * kAtQ + (row & 63);
    const int y = s * (kAtK / 2) + (kk >> 1);
    const int p = kk & 1;
    float v = 0.0f;
    if (q < (int64_t)g.nx * g.nz && y < g.ny) {
        const int64_t x = q % g.nx, z = q / g.nx;
        const int64_t pix = (z * g.ny + y) * g.nx + x;
        const float gq = G[pix];
        const float2 h = make_float2(gq * amp[2 * pix], -gq * amp[2 * pix + 1]);
        const bool im_row = (kind & 1) != 0;
        v = p == 0 ? (im_row ? h.y : h.x) : (im_row ? h.x : -h.y);
        if (kind >= 2) v *= (float)(g.ny0 + y);
    }
    uint16_t hi, lo;
    at_split(v, hi, lo);
    uint8_t* base = img + blk * kAtBBytes + at_chunk_mn(row, kk) + (uint32_t)(row & 7) * 2u;
    *reinterpret_cast<uint16_t*>(base) = hi;
    *reinterpret_cast<uint16_t*>(base + kAtBHalf) = lo;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kAtThreads, 1)
adjoint_tc_kernel(const AtomRec* __restrict__ rec, int64_t n_pad, GridDesc g, const uint8_t* __restrict__ img,
                  int n_rt, int n_st, int64_t n_work, float* __restrict__ partial, int* err, int64_t timeout_ns,
                  int64_t img_bytes, int64_t partial_n) {
    // img_bytes and partial_n (the sizes of `img` and `partial` the host
    // reserved) are read by the bounds checks of the checked build only
    extern __shared__ __align__(16) uint8_t at_raw[];
    const uint32_t raw = at_smem_u32(at_raw);
    uint8_t* smem = at_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t stage_base = at_smem_u32(smem);
    AtCtl* ctl = reinterpret_cast<AtCtl*>(smem + kAtStages * kAtStage);
    volatile int* abort_flag = &ctl->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = at_rank();  // 0: issues the MMAs of the pair
    const int64_t pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;

    // exp(i 2 pi k / 256): FP64 sincospi on the first octant (k <= 32) only,
    // the rest by the exact symmetries exp(i(pi/2 - t)) = i conj(exp(i t)) and
    // exp(i(t + pi/2)) = i exp(i t).  FP64 runs at a small fraction of the
    // FP32 rate, and 33 evaluations instead of 256 shorten the kernel's start.
    constexpr int kOct = kAtTab / 8, kQuad = kAtTab / 4;
    if (tid <= kOct) {
        double s, c;
        sincospi((double)tid / (kAtTab / 2), &s, &c);
        ctl->tab[tid] = make_float2((float)c, (float)s);
    }
    __syncthreads();
    for (int i = tid; i < kAtTab; i += kAtThreads) {
        if (i <= kOct) continue;
        const int q = i / kQuad, r = i % kQuad;
        float2 v = ctl->tab[r <= kOct ? r : kQuad - r];
        if (r > kOct) v = make_float2(v.y, v.x);
        for (int k = 0; k < q; ++k) v = make_float2(-v.y, v.x);
        ctl->tab[i] = v;
    }
    if (tid == kAtMmaWarp * 32) {
        for (int s = 0; s < kAtStages; ++s) {
            at_mbar_init(&ctl->full[s], kAtProdWarps + 1);
            at_mbar_init(&ctl->fill[s], kAtProdWarps);
            at_mbar_init(&ctl->copy[s], 1);
            at_mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            at_mbar_init(&ctl->acc_full[b], 1);
            at_mbar_init(&ctl->acc_empty[b], 2 * kAtEpiWarps);
        }
        at_mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kAtMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         at_smem_u32(&ctl->tmem)),
                     "r"(kAtTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    at_fence_before();
    at_cluster_sync();  // barriers of both CTAs initialised, tensor memory allocated
    at_fence_after();
    const uint32_t tmem = ctl->tmem;
    const int64_t Q = (int64_t)g.nx * g.nz;

    if (warp >= kAtProdWarp0) {
        // ------------------------------------------------------------ producers
        // warp w: atoms [32 (w & 3), +32) of the CTA, n_y [16 (w >> 2), +16) of the stage
        const int w = warp - kAtProdWarp0;
        const int a_loc = 32 * (w & 3) + lane;
        const int h = w >> 2;
        const uint32_t row_off = (uint32_t)(a_loc >> 3) * 1024u + (uint32_t)(a_loc & 7) * 128u;
        int slot = 0;
        uint32_t phase = 0;
        bool stop = false;
        for (int64_t wk = pair; wk < n_work && !stop; wk += n_pairs) {
            const int64_t tile = wk / n_rt;
            const int64_t j = tile * (2 * kAtAtomsCta) + (int64_t)rank * kAtAtomsCta + a_loc;
            const uint32_t U = j < n_pad ? __ldg(&rec[j].uy) : 0u;
            const float2 zstep = at_cis(U, ctl->tab);
            for (int s = 0; s < n_st && !stop; ++s) {
                const int y0 = s * (kAtK / 2) + 16 * h;  // local n_y of this thread's first value
                float2 E = at_cis((uint32_t)(g.ny0 + y0) * U, ctl->tab);
                if (!at_wait(&ctl->empty[slot], phase ^ 1u, abort_flag, err, timeout_ns)) {
                    stop = true;
                    break;
                }
                const uint32_t a_hi = stage_base + (uint32_t)slot * kAtStage + row_off;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // chunk 4h + c: k' = 8 (4h + c) .. +8, i.e. n_y y0 + 4c .. +4 as (Re, Im) pairs
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 v = (y0 + 4 * c + e < g.ny) ? E : make_float2(0.0f, 0.0f);
                        at_split2(v, hi[e], lo[e]);
                        E = at_cmul(E, zstep);
                    }
                    const uint32_t ch = (uint32_t)(((4 * h + c) ^ (a_loc & 7)) << 4);
                    if (XS_IN_BOUNDS(err, slot < kAtStages && row_off + ch + 16u <= kAtAHalf)) {
                        at_st_v4(a_hi + ch, hi[0], hi[1], hi[2], hi[3]);
                        at_st_v4(a_hi + kAtAHalf + ch, lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) at_arrive_local(rank == 0 ? &ctl->full[slot] : &ctl->fill[slot]);
                if (++slot == kAtStages) {
                    slot = 0;
                    phase ^= 1u;
                }
            }
        }
    } else if (warp == kAtLoadWarp) {
        // ------------------------------------------------------------ loader
        if (lane == 0) {
            int slot = 0;
            uint32_t phase = 0;
            uint32_t issued = 0u;  // bit s: a copy into slot s was issued (its latest phase)
            uint32_t last_par = 0u;
            bool stop = false;
            for (int64_t wk = pair; wk < n_work && !stop; wk += n_pairs) {
                const int rt = (int)(wk % n_rt);
                for (int s = 0; s < n_st && !stop; ++s) {
                    if (!at_wait(&ctl->empty[slot], phase ^ 1u, abort_flag, err, timeout_ns)) {
                        stop = true;
                        break;
                    }
                    const int64_t src_off = (((int64_t)rt * n_st + s) * 2 + rank) * kAtBBytes;
                    const uint8_t* src = img + src_off;
                    if (XS_IN_BOUNDS(err, slot < kAtStages && src_off >= 0 && src_off + kAtBBytes <= img_bytes)) {
                        at_arrive_expect_tx(&ctl->copy[slot], kAtBBytes);
                        at_bulk_copy(stage_base + (uint32_t)slot * kAtStage + 2 * kAtAHalf, src, kAtBBytes,
                                     &ctl->copy[slot]);
                    } else {
                        at_arrive_expect_tx(&ctl->copy[slot], 0u);  // completes the phase with no copy
                    }
                    issued |= 1u << slot;
                    last_par = (last_par & ~(1u << slot)) | (phase << slot);
                    if (++slot == kAtStages) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
            // the CTA leaves only after its copies have landed (bounded wait)
            int no_abort = 0;
            for (int s2 = 0; s2 < kAtStages; ++s2)
                if ((issued >> s2) & 1u) at_wait(&ctl->copy[s2], (last_par >> s2) & 1u, &no_abort, err, 2000000000LL);
        }
        __syncwarp();
    } else if (warp == kAtMmaWarp) {
        // ------------------------------------------------------------ MMA issue / relay
        if (rank == 0 && lane == 0) {
            constexpr uint32_t idesc = at_idesc(2 * kAtAtomsCta, kAtN);
            int slot = 0;
            uint32_t phase = 0;
            int64_t a_cnt = 0;
            bool ok = true;
            for (int64_t wk = pair; wk < n_work && ok; wk += n_pairs, ++a_cnt) {
                {
                    const int b = (int)(a_cnt & 1);
                    const uint32_t use = (uint32_t)(a_cnt >> 1);
                    if (!at_wait(&ctl->acc_empty[b], (use & 1u) ^ 1u, abort_flag, err, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    at_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)b * (uint32_t)kAtN;
                    for (int s = 0; s < n_st; ++s) {
                        if (!at_wait(&ctl->full[slot], phase, abort_flag, err, timeout_ns) ||
                            !at_wait(&ctl->copy[slot], phase, abort_flag, err, timeout_ns)) {
                            ok = false;
                            break;
                        }
                        at_fence_after();
                        const uint32_t a_hi = stage_base + (uint32_t)slot * kAtStage;
                        const uint32_t a_lo = a_hi + kAtAHalf;
                        const uint32_t b_hi = a_hi + 2 * kAtAHalf;
                        const uint32_t b_lo = b_hi + kAtBHalf;
                        if (XS_IN_BOUNDS(err, slot < kAtStages && (uint32_t)(b + 1) * kAtN <= kAtTmemCols)) {
#pragma unroll
                            for (int kk = 0; kk < kAtK / 16; ++kk) {
                                const uint32_t ka = (uint32_t)kk * 32u;    // K-major: 16 BF16 along the row
                                const uint32_t kb = (uint32_t)kk * 2048u;  // MN-major: two 8-row K atoms
                                at_mma_pair(d_tmem, at_desc_k(a_hi + ka), at_desc_mn(b_hi + kb), idesc,
                                            (s > 0 || kk > 0) ? 1u : 0u);
                                at_mma_pair(d_tmem, at_desc_k(a_hi + ka), at_desc_mn(b_lo + kb), idesc, 1u);
                                at_mma_pair(d_tmem, at_desc_k(a_lo + ka), at_desc_mn(b_hi + kb), idesc, 1u);
                            }
                        }
                        at_commit_pair(&ctl->empty[slot], 0x3);
                        if (++slot == kAtStages) {
                            slot = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) at_commit_pair(&ctl->acc_full[b], 0x3);
                }
            }
            // every issued MMA must finish before tensor memory is released
            at_commit_pair(&ctl->drain, 0x1);
            int no_abort = 0;
            at_wait(&ctl->drain, 0u, &no_abort, err, 2000000000LL);
        } else if (rank == 1 && lane == 0) {
            // relay: when this CTA's producers and copy have filled a stage,
            // arrive on CTA 0's full barrier with a cluster-scope release
            const uint32_t full_c0 = at_map(at_smem_u32(&ctl->full[0]), 0);
            int slot = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t wk = pair; wk < n_work && ok; wk += n_pairs) {
                for (int s = 0; s < n_st; ++s) {
                    if (!at_wait(&ctl->fill[slot], phase, abort_flag, err, timeout_ns) ||
                        !at_wait(&ctl->copy[slot], phase, abort_flag, err, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    at_arrive_cluster(full_c0 + (uint32_t)slot * 8u);
                    if (++slot == kAtStages) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        // TMEM lane quarter warp % 4 (a warp may only read its own quarter);
        // lane = atom of this CTA
        const int quarter = warp & 3;
        const int a_loc = 32 * quarter + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        const uint32_t acc_empty_c0 = at_map(at_smem_u32(&ctl->acc_empty[0]), 0);
        int64_t a_cnt = 0;
        for (int64_t wk = pair; wk < n_work; wk += n_pairs, ++a_cnt) {
            const int64_t tile = wk / n_rt;
            const int rt = (int)(wk % n_rt);
            const int64_t j = tile * (2 * kAtAtomsCta) + (int64_t)rank * kAtAtomsCta + a_loc;
            AtomRec me;
            me.ux = me.uy = me.uz = 0u;
            me.f = 0.0f;
            if (j < n_pad) me = rec[j];
            const float2 zx = at_cis(me.ux, ctl->tab);
            float tx = 0.0f, ty = 0.0f, tz = 0.0f;  // Im T of this thread's atom over the row tile
            const int b = (int)(a_cnt & 1);
            const uint32_t use = (uint32_t)(a_cnt >> 1);
            uint32_t got = 0;
            if (lane == 0) got = at_wait(&ctl->acc_full[b], use & 1u, abort_flag, err, timeout_ns, 200000u);
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) break;
            at_fence_after();
            const uint32_t dcol = lane_base + (uint32_t)b * (uint32_t)kAtN;
#pragma unroll 1
            for (int gq = 0; gq < kAtQ / 16; ++gq) {
                uint32_t rz[16], iz[16], ryv[16], iyv[16];
                if (XS_IN_BOUNDS(err, (uint32_t)b * kAtN + 3u * kAtQ + 16u * (gq + 1) <= kAtTmemCols)) {
                    at_ld16(dcol + 0 * kAtQ + 16 * gq, rz);
                    at_ld16(dcol + 1 * kAtQ + 16 * gq, iz);
                    at_ld16(dcol + 2 * kAtQ + 16 * gq, ryv);
                    at_ld16(dcol + 3 * kAtQ + 16 * gq, iyv);
                    at_wait_ld(rz);
                    at_wait_ld(iz);
                    at_wait_ld(ryv);
                    at_wait_ld(iyv);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) rz[i] = iz[i] = ryv[i] = iyv[i] = 0u;
                }
                const int64_t q0 = (int64_t)rt * kAtQ + 16 * gq;
                int xq = (int)(q0 % g.nx), zq = (int)(q0 / g.nx);
                float2 E = at_cis((uint32_t)(g.nx0 + xq) * me.ux + (uint32_t)(g.nz0 + zq) * me.uz, ctl->tab);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    if (q0 + i < Q) {
                        const float nxv = (float)(g.nx0 + xq), nzv = (float)(g.nz0 + zq);
                        // Im[E X] = Re E Im X + Im E Re X
                        const float ez = fmaf(E.x, __uint_as_float(iz[i]), E.y * __uint_as_float(rz[i]));
                        tx = fmaf(nxv, ez, tx);
                        tz = fmaf(nzv, ez, tz);
                        ty += fmaf(E.x, __uint_as_float(iyv[i]), E.y * __uint_as_float(ryv[i]));
                    }
                    // next row: n_x + 1, or the next n_z plane (reseeded)
                    if (++xq == g.nx) {
                        xq = 0;
                        ++zq;
                        E = at_cis((uint32_t)g.nx0 * me.ux + (uint32_t)(g.nz0 + zq) * me.uz, ctl->tab);
                    } else {
                        E = at_cmul(E, zx);
                    }
                }
            }
            at_fence_before();
            __syncwarp();
            if (lane == 0) at_arrive_cluster(acc_empty_c0 + (uint32_t)b * 8u);
            // this unit's sums of the atom: [unit][256 atoms][3]
            const int64_t pi = (wk * (2 * kAtAtomsCta) + (int64_t)rank * kAtAtomsCta + a_loc) * 3;
            if (XS_IN_BOUNDS(err, pi >= 0 && pi + 3 <= partial_n)) {
                float* pw = partial + pi;
                pw[0] = tx;
                pw[1] = ty;
                pw[2] = tz;
            }
        }
    }

    __syncwarp();
    at_fence_before();
    at_cluster_sync();  // no CTA leaves while the pair's MMAs or its peer may still touch it
    at_fence_after();
    if (warp == kAtMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAtTmemCols)
                     : "memory");
}

// one thread per atom: the row tiles' sums in row-tile order, then
// dL/dr_j = -4 pi f_j h^-T Im T_j
__global__ void adjoint_finish_kernel(const AtomRec* __restrict__ rec, int64_t n_atoms, int n_rt, Mat3 hinv,
                                      const float* __restrict__ partial, float* __restrict__ grad, int64_t partial_n,
                                      int* err) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n_atoms) return;
    const int64_t tile = j / (2 * kAtAtomsCta), jl = j % (2 * kAtAtomsCta);
    float t[3] = {0.0f, 0.0f, 0.0f};
    for (int rt = 0; rt < n_rt; ++rt) {
        const int64_t pi = (((tile * n_rt + rt) * (2 * kAtAtomsCta)) + jl) * 3;
        if (!XS_IN_BOUNDS(err, pi + 3 <= partial_n)) continue;
        const float* p = partial + pi;
        t[0] += p[0];
        t[1] += p[1];
        t[2] += p[2];
    }
    const double scale = -4.0 * 3.14159265358979323846 * (double)rec[j].f;
    for (int c = 0; c < 3; ++c) {
        const double hv = hinv.a[0 * 3 + c] * t[0] + hinv.a[1 * 3 + c] * t[1] + hinv.a[2 * 3 + c] * t[2];
        grad[j * 3 + c] = (float)(scale * hv);
    }
}

}  // namespace

static size_t image_bytes(const GridDesc& g) {
    const int64_t n_rt = ((int64_t)g.nx * g.nz + kAtQ - 1) / kAtQ;
    const int64_t n_st = ((int64_t)g.ny + kAtK / 2 - 1) / (kAtK / 2);
    return (size_t)(n_rt * n_st) * 2 * kAtBBytes;
}

size_t adjoint_tc_image_bytes(const GridDesc& g, int64_t n_pad) {
    const int64_t n_rt = ((int64_t)g.nx * g.nz + kAtQ - 1) / kAtQ;
    const int64_t n_tiles = (n_pad + 2 * kAtAtomsCta - 1) / (2 * kAtAtomsCta);
    return image_bytes(g) + (size_t)(n_tiles * n_rt) * (2 * kAtAtomsCta) * 3 * sizeof(float);
}

cudaError_t launch_adjoint_tc(const AtomRec* rec, int64_t n_atoms, int64_t n_pad, const GridDesc& g,
                              const Mat3& hinv, const float* amp, const float* G, void* image, float* grad, int* err,
                              int64_t timeout_ns, cudaStream_t st) {
    const int64_t n_rt = ((int64_t)g.nx * g.nz + kAtQ - 1) / kAtQ;
    const int64_t n_st = ((int64_t)g.ny + kAtK / 2 - 1) / (kAtK / 2);
    if (n_rt * n_st > INT32_MAX / 2) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(image) & 15u) != 0) return cudaErrorInvalidValue;  // bulk copies
    uint8_t* img = static_cast<uint8_t*>(image);
    const int64_t n_el = n_rt * n_st * 2 * 128 * kAtK;
    ++tl_kernel_launches;
    adjoint_image_kernel<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(amp, G, g, (int)n_rt, (int)n_st, img);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(adjoint_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAtSmemBytes);
    if (e != cudaSuccess) return e;
    // pairs resident at once (a cluster needs two SMs of one GPC), persistent
    // over the 256-atom tiles
    static int max_pairs = -1;
    if (max_pairs < 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (unsigned)std::max(1, sms / 2), 1, 1);
        cfg.blockDim = dim3(kAtThreads, 1, 1);
        cfg.dynamicSmemBytes = kAtSmemBytes;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 2;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (const void*)adjoint_tc_kernel, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = std::max(1, sms / 2);
        }
        max_pairs = n;
    }
    const int64_t n_tiles = (n_pad + 2 * kAtAtomsCta - 1) / (2 * kAtAtomsCta);
    const int64_t n_work = n_tiles * n_rt;  // units (atom tile, row tile)
    const int64_t pairs = std::min<int64_t>(max_pairs, n_work);
    float* partial = reinterpret_cast<float*>(img + image_bytes(g));
    const int64_t img_bytes = (int64_t)image_bytes(g);
    const int64_t partial_n = (int64_t)((adjoint_tc_image_bytes(g, n_pad) - image_bytes(g)) / sizeof(float));
    ++tl_kernel_launches;
    adjoint_tc_kernel<<<(unsigned)(2 * pairs), kAtThreads, kAtSmemBytes, st>>>(rec, n_pad, g, img, (int)n_rt,
                                                                              (int)n_st, n_work, partial, err,
                                                                              timeout_ns, img_bytes, partial_n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++tl_kernel_launches;
    adjoint_finish_kernel<<<(unsigned)((n_atoms + 255) / 256), 256, 0, st>>>(rec, n_atoms, (int)n_rt, hinv, partial,
                                                                             grad, partial_n, err);
    return cudaGetLastError();
}

}  // namespace xs
