// Tensor-core form of the direct method (Algorithm 1, Sec. 3.1).
//
// For q on the reciprocal lattice (q = 2 pi h^-T n, Sec. 3.1) the phase of
// atom j factorises over the axes:
//   exp(i q.r_j) = E_x[n_x](j) E_y[n_y](j) E_z[n_z](j),  E_a[n](j) = exp(i 2 pi n s_ja),
// so the amplitude of one detector plane is a complex contraction over atoms
//   S(n_x, n_y) = sum_j E_x[n_x](j) * w_j(n_y),   w_j(n_y) = f_j E_z[n_z](j) E_y[n_y](j).
// With A = [Re E_x ; Im E_x] (rows) and B = [Re w ; Im w] (columns) the real
// product D = A B^T holds the four real partial sums, and
//   Re S = D[Re x][Re y] - D[Im x][Im y],  Im S = D[Re x][Im y] + D[Im x][Re y].
//
// One CTA owns a tile of 64 n_x by 128 n_y of one frame and plane
// (MMA M = 128, N = 256) and loops over all atoms 64 at a time:
//   * 6 producer warps build the factor tables straight into shared memory in
//     the 128-byte-swizzled K-major layout the tensor core reads: each
//     complex factor c is split into hi = RN(c) and lo = RN(c - hi) (FP16 or
//     BF16).  Phases come from 32-bit exact turn counts (n*U mod 2^32); a
//     seed exp(i 2 pi n0 U) per run of 8 n is advanced by the exact step
//     exp(i 2 pi U) in FP32.
//   * 1 thread issues tcgen05.mma (hi*hi + hi*lo + lo*hi, FP32 accumulate)
//     into tensor memory; every `chunk_stages` stages the partial sums go to a
//     second TMEM region, so no FP32 accumulator sums more than one chunk of
//     atoms before it is added to the running total.
//   * 4 epilogue warps add chunk sums into the running total in TMEM and, at
//     the end of a tile, recombine the quadrants into S and I = |S|^2.
// Every wait is bounded: on expiry the kernel sets the device error word and
// all roles leave their loops; tensor memory is released in every case.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kBM = 128;   // MMA M: 64 complex n_x as Re/Im rows
constexpr int kBN = 256;   // MMA N: 128 complex n_y as Re/Im columns
constexpr int kBK = 64;    // atoms per stage = one 128-byte swizzle row of 16-bit values
constexpr int kStages = 2;
constexpr int kTileX = 64;
constexpr int kTileY = 128;
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kProdWarps = 6;
constexpr int kProdThreads = kProdWarps * 32;
constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;
constexpr uint32_t kABytes = kBM * kBK * 2;
constexpr uint32_t kBBytes = kBN * kBK * 2;
constexpr uint32_t kStageBytes = 2 * kABytes + 2 * kBBytes;
constexpr uint32_t kTmemCols = 512;  // [0,256): chunk accumulator, [256,512): running total
constexpr uint32_t kSumCol = 256;

struct StageScratch {
    uint32_t ux[kBK];
    uint32_t uy[kBK];
    float2 zx[kBK];
    float2 zy[kBK];
    float2 w[kBK];
};

struct SmemCtl {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t acc_full;
    uint64_t acc_empty;
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

constexpr size_t kSmemBytes = 1024 + kStages * kStageBytes + kStages * sizeof(StageScratch) + sizeof(SmemCtl);

struct TcArgs {
    const uint4* rec;
    int64_t n_pad;
    int n_frames;
    GridDesc g;
    int tiles_x, tiles_y;
    int64_t n_units;
    int n_stages;
    int chunk_stages;
    float* I;
    float* amp;
    int* err;
    int64_t timeout_ns;
};

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major; accumulate unless acc == 0
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                     uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on `bar` once every tcgen05 operation issued so far by this thread completes
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 columns of this warp's 32 TMEM lanes; the registers are valid only after
// tmem_wait16 on them (which carries the data dependency for the compiler)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// waits for every outstanding tcgen05.ld of the thread; ties `r` to the wait
__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// orders later uses of `r` after a preceding tmem_wait16 (no instruction)
__device__ __forceinline__ void tmem_dep16(uint32_t* r) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// OR of `pred` over the 192 producer threads (named barrier 1)
__device__ __forceinline__ bool producers_any(bool pred) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((uint32_t)pred), "n"(kProdThreads)
        : "memory");
    return out != 0;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the leading-byte offset is unused in this layout).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 D, A and B FP16 (or BF16), both K-major.
__host__ __device__ constexpr uint32_t make_idesc(bool bf16, int M, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// bounded wait; false if aborted or timed out (which also raises the abort flag)
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    uint32_t it = 0;
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((++it & 63u) == 0 && (int64_t)(globaltimer_ns() - t0) > timeout_ns) {
            *abort_flag = 1;
            set_dev_error(err, kDevErrTimeout);
            return false;
        }
    }
}

// ---- table construction ------------------------------------------------------

template <bool BF16>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// Writes the 8 atoms of one 16-byte chunk of `row` (hi and lo tiles).
template <bool BF16>
__device__ __forceinline__ void put_chunk(uint32_t hi_base, uint32_t lo_base, int row, int chunk, const float* v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split2<BF16>(v[2 * j], v[2 * j + 1], h[j], l[j]);
    const uint32_t off = (uint32_t)row * 128u + ((uint32_t)(chunk ^ (row & 7)) << 4);
    st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
    st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

struct UnitPos {
    int t, iz, tx, ty;
};

__device__ __forceinline__ UnitPos decode_unit(int64_t u, const TcArgs& a) {
    UnitPos p;
    p.tx = (int)(u % a.tiles_x);
    int64_t r = u / a.tiles_x;
    p.ty = (int)(r % a.tiles_y);
    r /= a.tiles_y;
    p.iz = (int)(r % a.g.nz);
    p.t = (int)(r / a.g.nz);
    return p;
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) tc_kernel(TcArgs args) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* smem = smem_raw + pad;
    const uint32_t stage_base = smem_u32(smem);
    StageScratch* scratch = reinterpret_cast<StageScratch*>(smem + kStages * kStageBytes);
    SmemCtl* ctl = reinterpret_cast<SmemCtl*>(smem + kStages * kStageBytes + kStages * sizeof(StageScratch));
    volatile int* abort_flag = &ctl->abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == kMmaWarp * 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&ctl->full[s], kProdThreads);
            mbar_init(&ctl->empty[s], 1);
        }
        mbar_init(&ctl->acc_full, 1);
        mbar_init(&ctl->acc_empty, kEpiWarps * 32);
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&ctl->tmem_base, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    const int64_t my_units =
        args.n_units > blockIdx.x ? (args.n_units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int n_chunks = (args.n_stages + args.chunk_stages - 1) / args.chunk_stages;

    if (warp >= kMmaWarp + 1) {
        // ------------------------------------------------------------ producers
        const int pt = threadIdx.x - (kMmaWarp + 1) * 32;
        const bool is_a = pt < 64;
        const int v = is_a ? pt : pt - 64;
        const int ag = v & 7;   // 16-byte chunk = atoms [8ag, 8ag+8) of the stage
        const int nr = v >> 3;  // run of 8 consecutive n (A: 0..7, B: 0..15)
        const int64_t total = my_units * args.n_stages;
        const bool loader = pt < 2 * kBK;
        const int la = pt & (kBK - 1);
        auto rec_addr = [&](int64_t L) -> const uint4* {
            const int64_t k = L / args.n_stages;
            const int s = (int)(L - k * args.n_stages);
            const int64_t u = blockIdx.x + k * gridDim.x;
            const UnitPos up = decode_unit(u, args);
            return args.rec + (int64_t)up.t * args.n_pad + (int64_t)s * kBK + la;
        };
        uint4 r_next = make_uint4(0, 0, 0, 0);
        if (loader && total > 0) r_next = __ldg(rec_addr(0));
        bool failed = false;
        for (int64_t L = 0; L < total; ++L) {
            const int slot = (int)(L & 1);
            const uint32_t round = (uint32_t)(L >> 1);
            const int64_t k = L / args.n_stages;
            const UnitPos up = decode_unit(blockIdx.x + k * gridDim.x, args);
            StageScratch* sc = &scratch[slot];
            if (loader) {
                const uint4 r = r_next;
                if (L + 1 < total) r_next = __ldg(rec_addr(L + 1));
                float c, s;
                if (pt < kBK) {
                    sc->ux[la] = r.x;
                    phase_to_cs(r.x, c, s);
                    sc->zx[la] = make_float2(c, s);
                } else {
                    sc->uy[la] = r.y;
                    phase_to_cs(r.y, c, s);
                    sc->zy[la] = make_float2(c, s);
                    const float f = __uint_as_float(r.w);
                    phase_to_cs((uint32_t)(args.g.nz0 + up.iz) * r.z, c, s);
                    sc->w[la] = make_float2(f * c, f * s);
                }
            }
            if (producers_any(failed || *abort_flag)) break;
            if (!wait_bar(&ctl->empty[slot], (round & 1u) ^ 1u, abort_flag, args.err, args.timeout_ns)) {
                failed = true;
                continue;
            }
            const uint32_t sb = stage_base + (uint32_t)slot * kStageBytes;
            float2 E[8], z[8];
            if (is_a) {
                const uint32_t n0 = (uint32_t)(args.g.nx0 + up.tx * kTileX + nr * 8);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float c, s;
                    phase_to_cs(n0 * sc->ux[8 * ag + i], c, s);
                    E[i] = make_float2(c, s);
                    z[i] = sc->zx[8 * ag + i];
                }
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int xi = nr * 8 + kk;
                    const int row_re = 32 * (xi >> 4) + (xi & 15);
                    float vr[8], vi[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        vr[i] = E[i].x;
                        vi[i] = E[i].y;
                    }
                    put_chunk<BF16>(sb, sb + kABytes, row_re, ag, vr);
                    put_chunk<BF16>(sb, sb + kABytes, row_re + 16, ag, vi);
                    if (kk < 7) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) E[i] = cmul(E[i], z[i]);
                    }
                }
            } else {
                const uint32_t n0 = (uint32_t)(args.g.ny0 + up.ty * kTileY + nr * 8);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float c, s;
                    phase_to_cs(n0 * sc->uy[8 * ag + i], c, s);
                    E[i] = cmul(sc->w[8 * ag + i], make_float2(c, s));
                    z[i] = sc->zy[8 * ag + i];
                }
                const uint32_t bh = sb + 2 * kABytes;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int m = nr * 8 + kk;
                    float vr[8], vi[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        vr[i] = E[i].x;
                        vi[i] = E[i].y;
                    }
                    put_chunk<BF16>(bh, bh + kBBytes, 2 * m, ag, vr);
                    put_chunk<BF16>(bh, bh + kBBytes, 2 * m + 1, ag, vi);
                    if (kk < 7) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) E[i] = cmul(E[i], z[i]);
                    }
                }
            }
            fence_async_shared();
            mbar_arrive(&ctl->full[slot]);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            constexpr uint32_t idesc = make_idesc(BF16, kBM, kBN);
            int64_t L = 0, a_cnt = 0;
            bool ok = true;
            for (int64_t k = 0; k < my_units && ok; ++k) {
                for (int c = 0; c < n_chunks && ok; ++c, ++a_cnt) {
                    if (!wait_bar(&ctl->acc_empty, ((uint32_t)a_cnt & 1u) ^ 1u, abort_flag, args.err,
                                  args.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (c == 0 ? kSumCol : 0u);
                    const int s0 = c * args.chunk_stages;
                    const int s1 = min(args.n_stages, s0 + args.chunk_stages);
                    for (int s = s0; s < s1; ++s, ++L) {
                        const int slot = (int)(L & 1);
                        const uint32_t round = (uint32_t)(L >> 1);
                        if (!wait_bar(&ctl->full[slot], round & 1u, abort_flag, args.err, args.timeout_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_hi = stage_base + (uint32_t)slot * kStageBytes;
                        const uint32_t a_lo = a_hi + kABytes;
                        const uint32_t b_hi = a_hi + 2 * kABytes;
                        const uint32_t b_lo = b_hi + kBBytes;
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint32_t ko = (uint32_t)kk * 32u;
                            umma(d_tmem, sw128_desc(a_hi + ko), sw128_desc(b_hi + ko), idesc,
                                 (s > s0 || kk > 0) ? 1u : 0u);
                            umma(d_tmem, sw128_desc(a_hi + ko), sw128_desc(b_lo + ko), idesc, 1u);
                            umma(d_tmem, sw128_desc(a_lo + ko), sw128_desc(b_hi + ko), idesc, 1u);
                        }
                        umma_commit(&ctl->empty[slot]);
                    }
                    if (ok) umma_commit(&ctl->acc_full);
                }
            }
            // every issued MMA must finish before tensor memory is released
            umma_commit(&ctl->drain);
            int dummy = 0;
            wait_bar(&ctl->drain, 0u, &dummy, args.err, args.timeout_ns);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const bool re_row = lane < 16;
        const int xi = warp * 16 + (lane & 15);
        int64_t a_cnt = 0;
        bool ok = true;
        for (int64_t k = 0; k < my_units && ok; ++k) {
            const UnitPos up = decode_unit(blockIdx.x + k * gridDim.x, args);
            for (int c = 0; c < n_chunks; ++c, ++a_cnt) {
                uint32_t got = 0;
                if (lane == 0)
                    got = wait_bar(&ctl->acc_full, (uint32_t)a_cnt & 1u, abort_flag, args.err, args.timeout_ns);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const bool last = c == n_chunks - 1;
                if (!last) {
                    if (c >= 1) {
#pragma unroll 1
                        for (int j = 0; j < kBN / 16; ++j) {
                            uint32_t d[16], sm[16];
                            tmem_ld16(lane_base + 16 * j, d);
                            tmem_ld16(lane_base + kSumCol + 16 * j, sm);
                            tmem_wait16(d);
                            tmem_dep16(sm);
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                sm[i] = __float_as_uint(__uint_as_float(sm[i]) + __uint_as_float(d[i]));
                            tmem_st16(lane_base + kSumCol + 16 * j, sm);
                        }
                        tmem_st_wait();
                    }
                } else {
                    const int ix = up.tx * kTileX + xi;
#pragma unroll 1
                    for (int j = 0; j < 8; ++j) {
                        uint32_t rlo[16], rhi[16];
                        float lo[16], hi[16];
                        tmem_ld16(lane_base + kSumCol + 16 * j, rlo);
                        tmem_ld16(lane_base + kSumCol + 128 + 16 * j, rhi);
                        if (c >= 1) {
                            uint32_t dl[16], dh[16];
                            tmem_ld16(lane_base + 16 * j, dl);
                            tmem_ld16(lane_base + 128 + 16 * j, dh);
                            tmem_wait16(rlo);
                            tmem_dep16(rhi);
                            tmem_dep16(dl);
                            tmem_dep16(dh);
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                lo[i] = __uint_as_float(rlo[i]) + __uint_as_float(dl[i]);
                                hi[i] = __uint_as_float(rhi[i]) + __uint_as_float(dh[i]);
                            }
                        } else {
                            tmem_wait16(rlo);
                            tmem_dep16(rhi);
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                lo[i] = __uint_as_float(rlo[i]);
                                hi[i] = __uint_as_float(rhi[i]);
                            }
                        }
                        float own[16], rcv[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            own[i] = re_row ? lo[i] : hi[i];
                            const float snd = re_row ? hi[i] : lo[i];
                            rcv[i] = __shfl_xor_sync(0xffffffffu, snd, 16);
                        }
                        if (ix < args.g.nx) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) {
                                const float p_rr = re_row ? own[2 * e] : rcv[2 * e];
                                const float p_ri = re_row ? own[2 * e + 1] : rcv[2 * e + 1];
                                const float p_ir = re_row ? rcv[2 * e] : own[2 * e];
                                const float p_ii = re_row ? rcv[2 * e + 1] : own[2 * e + 1];
                                const float sre = p_rr - p_ii;
                                const float sim = p_ri + p_ir;
                                const int m = (re_row ? 0 : 64) + 8 * j + e;
                                const int iy = up.ty * kTileY + m;
                                if (iy < args.g.ny) {
                                    const int64_t o =
                                        (((int64_t)up.t * args.g.nz + up.iz) * args.g.ny + iy) * args.g.nx + ix;
                                    args.I[o] = sre * sre + sim * sim;
                                    if (args.amp) {
                                        args.amp[2 * o] = sre;
                                        args.amp[2 * o + 1] = sim;
                                    }
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&ctl->acc_empty);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

bool tc_supported(const GridDesc& g) { return g.nx >= 1 && g.ny >= 1 && g.nz >= 1; }

TcPlan plan_tc(int64_t n_pad, int64_t n_frames, const GridDesc& g, int num_sms, int chunk_stages) {
    TcPlan p;
    p.tiles_x = (g.nx + kTileX - 1) / kTileX;
    p.tiles_y = (g.ny + kTileY - 1) / kTileY;
    const int64_t units = n_frames * g.nz * p.tiles_x * p.tiles_y;
    p.grid = (int)std::min<int64_t>(units, num_sms);
    p.chunk_stages = chunk_stages > 0 ? chunk_stages : 64;
    (void)n_pad;
    return p;
}

cudaError_t launch_tc(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g, const TcPlan& plan,
                      bool bf16, float* I, float* amp, int* err, int64_t timeout_ns, cudaStream_t st) {
    if (n_pad % kBK != 0) return cudaErrorInvalidValue;
    TcArgs a;
    a.rec = reinterpret_cast<const uint4*>(rec);
    a.n_pad = n_pad;
    a.n_frames = (int)n_frames;
    a.g = g;
    a.tiles_x = plan.tiles_x;
    a.tiles_y = plan.tiles_y;
    a.n_units = n_frames * g.nz * plan.tiles_x * plan.tiles_y;
    a.n_stages = (int)(n_pad / kBK);
    a.chunk_stages = plan.chunk_stages;
    a.I = I;
    a.amp = amp;
    a.err = err;
    a.timeout_ns = timeout_ns;
    if (a.n_units == 0) return cudaSuccess;
    const void* fn = bf16 ? (const void*)tc_kernel<true> : (const void*)tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    if (bf16)
        tc_kernel<true><<<plan.grid, kThreads, kSmemBytes, st>>>(a);
    else
        tc_kernel<false><<<plan.grid, kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace xs
