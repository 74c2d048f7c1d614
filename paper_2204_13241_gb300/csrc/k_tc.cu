// Tensor-core form of the direct method (Algorithm 1, Sec. 3.1).
//
// For q on the reciprocal lattice (q = 2 pi h^-T n, Sec. 3.1) the phase of
// atom j factorises over the axes:
//   exp(i q.r_j) = E_x[n_x](j) E_y[n_y](j) E_z[n_z](j),  E_a[n](j) = exp(i 2 pi n s_ja),
// so the amplitude of one detector plane is a complex contraction over atoms
//   S(n_x, n_y) = sum_j E_x[n_x](j) * w_j(n_y),   w_j(n_y) = f_j E_z[n_z](j) E_y[n_y](j).
// Rows of A are Re and Im of E_x[n_x], rows of B are Re and Im of w(n_y); within
// each group of 4 rows the order is (Re n, Re n+1, Im n, Im n+1) for even n.
// The real product D = A B^T holds the four real partial sums:
//   Re S = D[Re x][Re y] - D[Im x][Im y],  Im S = D[Re x][Im y] + D[Im x][Re y].
//
// A pair of CTAs (a cluster of two on neighbouring SMs) owns a tile of
// 128 n_x by 128 n_y of one frame and plane and runs one M = 256, N = 256
// tcgen05 contraction (cta_group::2) over all atoms, 64 atoms per stage.
// CTA r holds the A rows of n_x [64r, 64r+64) and the B rows of n_y
// [64r, 64r+64) of the tile, so each CTA builds only a quarter of the pair's
// factor tables; the accumulator rows of CTA r (in its own tensor memory) are
// its A rows against all 256 B columns.
//   * 8 producer warps per CTA write the tables straight into shared memory in
//     the MN-major, 128-byte-swizzled layout the tensor core reads.  Each
//     thread owns one atom and a run of consecutive n (32 or 16), held as
//     pairs (n, n+1) in packed FP32x2 registers: the run starts from the
//     seed exp(i 2 pi n0 U) of an exact turn count (U = 32-bit turn count,
//     n U mod 2^32 is exact) and z = exp(i 2 pi U), takes exp(i 2 pi (n0+1) U)
//     = seed z, and advances by the step z^2.  Each value
//     c is split into hi = RN(c) and lo = RN(c - hi) (FP16 or BF16).
//   * Producer warps arrive on a barrier of their own CTA (CTA-scope
//     release); in CTA 1 one relay thread forwards each filled stage to CTA 0
//     with a single cluster-scope release.
//   * 1 thread of CTA 0 issues tcgen05.mma (hi*hi + hi*lo + lo*hi, FP32
//     accumulate) into one of two TMEM accumulators; after `chunk_stages`
//     stages it hands the accumulator to the epilogues and continues in the
//     other one.
//   * 4 epilogue warps per CTA add each chunk's FP32 sums into running totals
//     kept as error-free FP32 pairs (hi + lo, updated by TwoSum) in an
//     L2-resident scratch block (one per CTA) and, after the last chunk of a
//     tile, recombine the quadrants in FP64 into S and I = |S|^2.
// On centred tiles (n_x, n_y in [-64, 64), n_z = 0) the tables use Friedel
// symmetry of the factors, E(-n) = conj E(n) and w(-n) = conj w(n) for real
// f: each CTA holds n in [32r, 32r + 32) and their negatives, builds 33 base
// values per operand instead of 64 and stores each twice (see centred_index).
// Units (frame x plane x tile) are dealt round-robin to the pairs.  When the
// last wave is partial, its units are cut along the atoms into pieces; each
// piece leaves its FP64 partial amplitude, and split_finish_kernel adds the
// pieces in part order after the launch.
// The atoms arrive in a coprime-stride permuted order (see the phase kernel),
// so the partial sums over a chunk behave like random walks even for ordered
// crystals and the FP32 accumulator never sums a coherent run of terms.
// Every wait is bounded: on expiry the kernel sets the device error word and
// all roles leave their loops; tensor memory is released in every case.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <queue>
#include <vector>

#include "xs_internal.h"

namespace xs {

namespace {

constexpr int kBK = 64;     // atoms per stage
constexpr int kTile = 128;  // n_x per pair tile (M of the pair: Re/Im rows of 128 n_x)
constexpr int kHalf = 64;   // n_x per CTA
constexpr int kEpiWarps = 4;
constexpr int kMmaWarp = 4;
constexpr int kMaxStages = 4;
// MN-major SW128 tiles: blocks of 64 MN elements (128-byte rows), 8 K rows per
// 1024-byte swizzle atom; a stage holds kBK / 8 = 8 K atoms per MN block.
constexpr uint32_t kMNBlockBytes = (kBK / 8) * 1024;  // 8 KB: leading byte offset
constexpr uint32_t kAHalfBytes = 2 * kMNBlockBytes;    // 128 A rows of one operand half

// The two tile kinds.  Per CTA the A side is always the Re/Im rows of 64 n_x
// and the B side the Re/Im rows of kTileY / 2 n_y; each producer thread owns
// one atom and a run of kRun consecutive n of one side.
template <int KIND>
struct Cfg;
template <>
struct Cfg<kTcTile128> {
    static constexpr int kTileY = 128;  // n_y per pair tile
    static constexpr int kBN = 256;     // MMA N: Re/Im columns of kTileY n_y
    static constexpr int kRun = 32;
    static constexpr int kStages = 3;
    static constexpr uint32_t kTmemCols = 512;  // two 256-column FP32 accumulators
};
template <>
struct Cfg<kTcTile64> {
    static constexpr int kTileY = 64;
    static constexpr int kBN = 128;
    static constexpr int kRun = 16;
    static constexpr int kStages = 4;
    static constexpr uint32_t kTmemCols = 256;  // two 128-column FP32 accumulators
};

struct SmemCtl {
    uint64_t full[kMaxStages];   // CTA 0: its producer warps and the peer's relay
    uint64_t fill[kMaxStages];   // CTA 1: its producer warps (forwarded by the relay)
    uint64_t empty[kMaxStages];  // each CTA: MMA commits
    uint64_t acc_full[2];     // each CTA: MMA commits
    uint64_t acc_empty[2];    // CTA 0: epilogue warps of both CTAs
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
    float2 tab[256];          // exp(i 2 pi k / 256)
};

template <int KIND>
struct Lay {
    using C = Cfg<KIND>;
    static constexpr int kARuns = kHalf / C::kRun;              // runs over the CTA's n_x
    static constexpr int kBRuns = (C::kTileY / 2) / C::kRun;    // runs over the CTA's n_y
    static constexpr int kProdWarps = 2 * (kARuns + kBRuns);    // two warps (32 atoms each) per run
    static constexpr int kThreads = (kEpiWarps + 1 + kProdWarps) * 32;
    static constexpr uint32_t kBHalfBytes = (uint32_t)(C::kTileY / 64) * kMNBlockBytes;
    static constexpr uint32_t kStageBytes = 2 * kAHalfBytes + 2 * kBHalfBytes;  // A hi, A lo, B hi, B lo
    static constexpr size_t kSmemBytes = 1024 + (size_t)C::kStages * kStageBytes + sizeof(SmemCtl);
    static_assert(C::kStages <= kMaxStages, "stage barriers");
    static_assert(kProdWarps * 32 + (kEpiWarps + 1) * 32 <= 1024, "block size");
};

struct TcArgs {
    TcTraj single;          // the trajectory when `units` is null
    // single trajectory: units [0, full * n_pairs) round-robin, whole; the
    // remaining `rem` units are split along the atoms into `parts` stage
    // ranges each, and the rem * parts pieces are dealt round-robin as well
    int64_t full, rem;
    int parts;
    const TcTraj* trajs;    // batched: trajectory table
    const int4* units;      // batched: (traj, frame, plane, tile_x | tile_y << 16), pair by pair
    const int* pair_start;  // batched: [n_pairs + 1] offsets into `units`
    int chunk_stages;
    double* scratch;        // [gridDim.x][256][128] running totals as FP32 pairs (hi, lo)
    double2* partial;       // split units: [rem][parts][128 x][128 y] partial amplitudes
    int* err;
    int64_t timeout_ns;
#ifdef XS_BOUNDS_CHECK
    int64_t scratch_f2;     // float2 entries of `scratch`
    int64_t partial_n;      // double2 entries of `partial`
#endif
};

// ---- PTX wrappers ------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// address of the same shared-memory object in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// arrive (release at cluster scope) on a barrier given by its cluster address
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

// arrive (release at CTA scope) on a barrier of this CTA
__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Test of the phase with parity `parity`; the thread may sleep in the barrier
// for up to `hint_ns` before the answer comes back (no busy issue slots).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
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

// one warp of each CTA of the pair allocates the same columns in both
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

// D[tmem of both CTAs] (+)= A[smem of both] * B[smem of both]^T (M = 256);
// accumulate unless acc == 0.  Issued by one thread of CTA 0.
__device__ __forceinline__ void umma_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on `bar` in the CTAs of `mask` once every tcgen05 operation issued so
// far by this thread completes
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
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

__device__ __forceinline__ void tmem_wait16(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// Shared-memory matrix descriptor, MN-major with 128-byte swizzle: leading
// byte offset = stride between 64-element MN blocks, stride byte offset =
// stride between 8-row K atoms (1024 B).
__device__ __forceinline__ uint64_t mn_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(kMNBlockBytes >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 D, A and B FP16 (or BF16), both MN-major.
__host__ __device__ constexpr uint32_t make_idesc(bool bf16, int M, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bounded wait; false if aborted or timed out (which also raises the abort flag)
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int64_t timeout_ns,
                         uint32_t hint_ns) {
    if (mbar_try_wait(bar, parity, 0u)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity, hint_ns)) return true;
        if (*abort_flag) return false;
        if ((int64_t)(globaltimer_ns() - t0) > timeout_ns) {
            *abort_flag = 1;
            set_dev_error(err, kDevErrTimeout);
            return false;
        }
    }
}

// ---- table construction ------------------------------------------------------

// exp(i 2 pi P / 2^32) for a 32-bit turn count: the top 8 bits pick
// exp(i 2 pi k / 256) from a table in shared memory, the remaining angle
// t < 2 pi / 256 uses the Taylor polynomials cos t = 1 - t^2/2 + t^4/24 and
// sin t = t - t^3/6 + t^5/120 (truncation below 3e-13), and the two factors
// are multiplied: about 15 instructions.  Evaluating the seeds in registers
// with sincospif of the top 24 bits instead took about twice the
// instructions and made the producer-bound tiles 2-5% slower.
__device__ __forceinline__ float2 cis_turns(uint32_t P, const float2* tab) {
    const float2 a = tab[P >> 24];
    const float t = (float)(P & 0xFFFFFFu) * 1.4629180792671596e-9f;  // 2 pi / 2^32
    const float t2 = t * t;
    const float c = fmaf(t2, fmaf(t2, 1.0f / 24.0f, -0.5f), 1.0f);
    const float s = t * fmaf(t2, fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
}

// v = (v0, v1) -> packed hi = (RN(v0), RN(v1)) and lo = (RN(v0 - hi0), RN(v1 - hi1));
// v - hi is exact in FP32, so hi + lo carries about twice the format's bits
template <bool BF16>
__device__ __forceinline__ void split2(float2 v, uint32_t& hi, uint32_t& lo) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        const float2 d = __ffma2_rn(__bfloat1622float2(h), make_float2(-1.0f, -1.0f), v);
        const __nv_bfloat162 l = __float22bfloat162_rn(d);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __float22half2_rn(v);
        const float2 d = __ffma2_rn(__half22float2(h), make_float2(-1.0f, -1.0f), v);
        const __half2 l = __float22half2_rn(d);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// The FP64 table builder (a test and measurement option): w exp(i 2 pi P / 2^32)
// from sincospi of the exact turn count in FP64, rounded once to FP32; w is
// the B side's weight f E_z (1 on the A side), also in FP64.
__device__ __forceinline__ float2 cis_exact(uint32_t P, double2 w) {
    double s, c;
    sincospi((double)P * 4.656612873077392578125e-10, &s, &c);  // 2^-31
    return make_float2((float)(c * w.x - s * w.y), (float)(c * w.y + s * w.x));
}

// entries n and n + 1 of a run as (Re n, Re n+1) and (Im n, Im n+1)
__device__ __forceinline__ void exact_pair(uint32_t n, uint32_t U, double2 w, float2& R, float2& Im) {
    const float2 a = cis_exact(n * U, w), b = cis_exact((n + 1u) * U, w);
    R = make_float2(a.x, b.x);
    Im = make_float2(a.y, b.y);
}

// byte offset of the 16-byte chunk holding MN rows [mn, mn+8) of K row k
__device__ __forceinline__ uint32_t chunk_off(int mn, int k) {
    return (uint32_t)(mn >> 6) * kMNBlockBytes + (uint32_t)(k >> 3) * 1024u + (uint32_t)(k & 7) * 128u +
           ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4);
}

// Centred tiles (n in [-64, 64) on both axes, n_z = 0) use E(-n) = conj E(n)
// and, with real f and E_z = 1, w(-n) = conj w(n).  CTA r holds the rows of
// n in [32r, 32r + 32) and of their negatives, so it builds the 33 base values
// X(32r + s), s = 0..32, of each operand and stores every one twice: slot s
// (s < 32) holds X(32r + s) for n = 32r + s; slot 32 + s (s = 1..31) holds the
// same X(32r + s) for n = -(32r + s), and slot 32 holds X(32r + 32) for
// n = -(32r + 32).  The mirrored slots keep X itself, so their Im rows carry
// the sign of conj; the epilogue applies it.
__device__ __forceinline__ int centred_index(int slot, int r, float& sign) {
    if (slot < 32) {
        sign = 1.0f;
        return 32 * r + slot + kHalf;
    }
    const int s = slot - 32;
    sign = -1.0f;
    return kHalf - 32 * r - (s == 0 ? 32 : s);
}

// one tile of one frame and plane, with what every role needs to work on it
struct Unit {
    const uint4* rec;  // records of the unit's frame
    float* I;
    float* amp;
    int nx0, nx, ny0, ny, nz0, nz;
    int t, iz, tx, ty;
    bool centred;  // tile n_x, n_y in [-64, 64) on the plane n_z = 0
    int s0, s1;    // stage range of this piece of the unit
    int split;     // split unit index, or -1 for a whole unit
    int part;
    int chunk;     // stages per accumulation chunk (0: the launch's)
    int tile_y;    // n_y per tile
#ifdef XS_BOUNDS_CHECK
    const uint4* rec_lo;  // the trajectory's records [rec_lo, rec_hi)
    const uint4* rec_hi;
    int64_t out_n;        // entries of I the check admits
#endif
};

__device__ __forceinline__ Unit make_unit(const TcTraj& tr, int t, int iz, int tx, int ty) {
    Unit u;
    u.rec = tr.rec + (int64_t)t * tr.n_pad;
    u.I = tr.I;
    u.amp = tr.amp;
    u.nx0 = tr.nx0;
    u.nx = tr.nx;
    u.ny0 = tr.ny0;
    u.ny = tr.ny;
    u.nz0 = tr.nz0;
    u.nz = tr.nz;
    u.t = t;
    u.iz = iz;
    u.tx = tx;
    u.ty = ty;
    u.tile_y = tc_tile_y(tr.kind);
    u.centred = tr.kind == kTcTile128 && tr.nx0 + tx * kTile == -kHalf && tr.ny0 + ty * u.tile_y == -kHalf &&
                tr.nz0 + iz == 0;
    u.s0 = 0;
    u.s1 = tr.n_stages;
    u.split = -1;
    u.part = 0;
    u.chunk = tr.chunk;
#ifdef XS_BOUNDS_CHECK
    u.rec_lo = tr.rec;
    u.rec_hi = tr.rec + (int64_t)tr.n_frames * tr.n_pad;
    u.out_n = (int64_t)tr.check_frames * tr.nz * tr.ny * tr.nx;
#endif
    return u;
}

// record `p` of unit `u`; the checked build tests that it lies in the
// trajectory's records and reads a zero record in place of one that does not
__device__ __forceinline__ uint4 load_rec(const Unit& u, const uint4* p, int* err) {
    if (!XS_IN_BOUNDS(err, p >= u.rec_lo && p < u.rec_hi)) return make_uint4(0u, 0u, 0u, 0u);
    return __ldg(p);
}

// A tile with at most kHalf valid n_x rows (a grid at most 64 wide, or the
// last tile of one): each CTA of the pair takes kHalf / 2 of them, and the A
// runs past those are not built.  The rows left unbuilt hold whatever the
// stage held; their products only reach accumulator rows the epilogue drops.
// Not for centred tiles, which have their own row order.
__device__ __forceinline__ bool unit_narrow(const Unit& u, bool centred) {
    return !centred && u.nx - u.tx * kTile <= kHalf;
}

__device__ __forceinline__ Unit single_unit(const TcTraj& tr, int64_t u) {
    const int tx = (int)(u % tr.tiles_x);
    int64_t r = u / tr.tiles_x;
    const int ty = (int)(r % tr.tiles_y);
    r /= tr.tiles_y;
    const int iz = (int)(r % tr.nz);
    return make_unit(tr, (int)(r / tr.nz), iz, tx, ty);
}

// piece k of `pair`: round-robin over a single trajectory (whole units, then
// the pieces of the split ones), or the pair's list
__device__ __forceinline__ Unit get_unit(const TcArgs& a, int64_t pair, int64_t n_pairs, int64_t k) {
    if (!a.units) {
        const TcTraj& tr = a.single;
        if (k < a.full) return single_unit(tr, pair + k * n_pairs);
        const int64_t i = pair + (k - a.full) * n_pairs;  // piece index among the split units
        const int64_t r = i / a.parts;
        Unit u = single_unit(tr, a.full * n_pairs + r);
        if (a.parts > 1) {
            const int q = (int)(i - r * a.parts);
            u.s0 = (int)((int64_t)q * tr.n_stages / a.parts);
            u.s1 = (int)((int64_t)(q + 1) * tr.n_stages / a.parts);
            u.split = (int)r;
            u.part = q;
        }
        return u;
    }
    const int4 w = a.units[a.pair_start[pair] + k];
    return make_unit(a.trajs[w.x], w.y, w.z, w.w & 0xFFFF, w.w >> 16);
}

__device__ __forceinline__ int64_t units_of_pair(const TcArgs& a, int64_t pair, int64_t n_pairs) {
    if (!a.units) {
        const int64_t pieces = a.rem * a.parts;
        return a.full + (pieces > pair ? (pieces - 1 - pair) / n_pairs + 1 : 0);
    }
    return a.pair_start[pair + 1] - a.pair_start[pair];
}

// Pieces of the split units of a single-trajectory launch: one thread per
// pixel of the tile sums the parts' FP64 partial amplitudes in part order and
// writes I (and the amplitude).  Runs after tc_kernel on the same stream.
__global__ void split_finish_kernel(TcArgs a, int64_t n_pairs) {
    const int64_t r = blockIdx.y;  // split unit
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= kTile * kTile) return;
    const int xi = pix / kTile, yi = pix - xi * kTile;
    const Unit up = single_unit(a.single, a.full * n_pairs + r);
    if (yi >= up.tile_y) return;
    const int ix = up.tx * kTile + xi, iy = up.ty * up.tile_y + yi;
    if (ix >= up.nx || iy >= up.ny) return;
    const double2* base = a.partial + (size_t)r * a.parts * (kTile * kTile) + pix;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < a.parts; ++q) {
        const double2 v = base[(size_t)q * (kTile * kTile)];
        re += v.x;
        im += v.y;
    }
    const int64_t o = (((int64_t)up.t * up.nz + up.iz) * up.ny + iy) * up.nx + ix;
    up.I[o] = (float)(re * re + im * im);
    if (up.amp) {
        up.amp[2 * o] = (float)re;
        up.amp[2 * o + 1] = (float)im;
    }
}

template <bool BF16, int KIND, bool EXACT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(Lay<KIND>::kThreads, 1) tc_kernel(TcArgs args) {
    using C = Cfg<KIND>;
    using L = Lay<KIND>;
    constexpr int kStages = C::kStages;
    constexpr uint32_t kStageBytes = L::kStageBytes;
    constexpr int kProdWarps = L::kProdWarps;
    constexpr int kRun = C::kRun;
    constexpr int kBN = C::kBN;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* smem = smem_raw + pad;
    const uint32_t stage_base = smem_u32(smem);
    SmemCtl* ctl = reinterpret_cast<SmemCtl*>(smem + kStages * kStageBytes);
    volatile int* abort_flag = &ctl->abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();  // 0: issues the MMAs of the pair
    const int64_t pair = blockIdx.x >> 1, n_pairs = gridDim.x >> 1;

    // exp(i 2 pi k / 256): FP64 sincospi on the first octant (k <= 32) only,
    // the rest by the exact symmetries exp(i(pi/2 - t)) = i conj(exp(i t)) and
    // exp(i(t + pi/2)) = i exp(i t) (FP64 runs at a small fraction of the
    // FP32 rate); the cluster barrier below orders the table for every warp
    if (threadIdx.x <= 32) {
        double sn, cs;
        sincospi((double)threadIdx.x / 128, &sn, &cs);
        ctl->tab[threadIdx.x] = make_float2((float)cs, (float)sn);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += L::kThreads) {
        if (i <= 32) continue;
        const int q = i >> 6, r = i & 63;
        float2 v = ctl->tab[r <= 32 ? r : 64 - r];
        if (r > 32) v = make_float2(v.y, v.x);
        for (int j = 0; j < q; ++j) v = make_float2(-v.y, v.x);
        ctl->tab[i] = v;
    }
    if (threadIdx.x == kMmaWarp * 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&ctl->full[s], kProdWarps + 1);
            mbar_init(&ctl->fill[s], kProdWarps);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->acc_full[b], 1);
            mbar_init(&ctl->acc_empty[b], 2 * kEpiWarps);
        }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc_pair(&ctl->tmem_base, C::kTmemCols);
    tc_fence_before();
    cluster_sync();  // barriers of both CTAs initialised, tensor memory allocated
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    const int64_t my_units = units_of_pair(args, pair, n_pairs);

    if (warp >= kMmaWarp + 1) {
        // ------------------------------------------------------------ producers
        // warp w: atoms [32 (w & 1), +32) of the stage; run ri = w >> 1: the
        // first kARuns runs cover the CTA's 64 n_x (A rows), the others its
        // kTileY / 2 n_y (B rows)
        const int w = warp - (kMmaWarp + 1);
        const int ri = w >> 1;
        const bool is_a = ri < L::kARuns;
        // general tiles: a run of kRun consecutive n of this CTA's half;
        // centred tiles (128 x 128 only): base values X(32 rank + s), s in
        // [s0, s0 + 16)
        const int run0 = kRun * (is_a ? ri : ri - L::kARuns);
        const int s0 = 16 * (ri & 1);
        const int k = 32 * (w & 1) + lane;
        int slot = 0;
        uint32_t phase = 0;  // parity of the current pass over the ring of stages
        Unit up{};
        if (my_units > 0) up = get_unit(args, pair, n_pairs, 0);
        uint4 r_next = make_uint4(0, 0, 0, 0);
        if (my_units > 0) r_next = load_rec(up, up.rec + (int64_t)up.s0 * kBK + k, args.err);
        bool stop = false;
        for (int64_t ku = 0; ku < my_units && !stop; ++ku) {
            Unit up_next{};
            const bool has_next = ku + 1 < my_units;
            if (has_next) up_next = get_unit(args, pair, n_pairs, ku + 1);
            const int st1 = up.s1;
            const uint4* rec_cur = up.rec + k;
            const bool centred = KIND == kTcTile128 && up.centred;
            const bool extra = centred && (ri & 1) == 0;  // also builds X(32 rank + 32)
            const bool narrow = unit_narrow(up, centred);
            const bool idle = is_a && narrow && run0 >= kHalf / 2;  // an A run past the narrow rows
            const uint32_t n0 =
                centred ? (uint32_t)(32 * (int)rank + s0)
                        : (is_a ? (uint32_t)(up.nx0 + up.tx * kTile + (narrow ? kHalf / 2 : kHalf) * (int)rank + run0)
                                : (uint32_t)(up.ny0 + up.ty * C::kTileY + (C::kTileY / 2) * (int)rank + run0));
            const uint32_t nz = (uint32_t)(up.nz0 + up.iz);
            for (int s = up.s0; s < st1; ++s) {
                const uint4 r = r_next;
                if (s + 1 < st1)
                    r_next = load_rec(up, rec_cur + (int64_t)(s + 1) * kBK, args.err);
                else if (has_next)
                    r_next = load_rec(up_next, up_next.rec + (int64_t)up_next.s0 * kBK + k, args.err);
                if (idle) {
                    // nothing to build: take the slot and pass it on
                    if (!wait_bar(&ctl->empty[slot], phase ^ 1u, abort_flag, args.err, args.timeout_ns, 20000u)) {
                        stop = true;
                        break;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive_local(rank == 0 ? &ctl->full[slot] : &ctl->fill[slot]);
                    if (++slot == kStages) {
                        slot = 0;
                        phase ^= 1u;
                    }
                    continue;
                }
                // seed E(n0) and z = E(1) of this thread's run, E(n0 + 1) = E(n0) z
                // and the step z^2 (two table evaluations instead of three
                // made producer-bound tiles 2-7% faster, at the same error)
                const uint32_t U = is_a ? r.x : r.y;
                const float2 z1 = cis_turns(U, ctl->tab);
                float2 E0 = cis_turns(n0 * U, ctl->tab);
                float2 E1 = cmul(E0, z1);
                const float2 z2 = cmul(z1, z1);
                const float2 ZR = make_float2(z2.x, z2.x), ZI = make_float2(z2.y, z2.y);
                const float2 NZI = make_float2(-z2.y, -z2.y);
                float2 Ex = make_float2(0.0f, 0.0f);
                if (extra) Ex = cis_turns((uint32_t)(32 * (int)rank + 32) * U, ctl->tab);
                double2 wd = make_double2(1.0, 0.0);  // the FP64 builder's weight
                if (!is_a) {
                    const float f = __uint_as_float(r.w);
                    float2 wv = make_float2(f, 0.0f);
                    if (nz != 0u) {
                        const float2 ez = cis_turns(nz * r.z, ctl->tab);
                        wv = make_float2(f * ez.x, f * ez.y);
                    }
                    E0 = cmul(E0, wv);
                    E1 = cmul(E1, wv);
                    Ex = cmul(Ex, wv);
                    if constexpr (EXACT) {
                        wd = make_double2((double)f, 0.0);
                        if (nz != 0u) {
                            double se, ce;
                            sincospi((double)(nz * r.z) * 4.656612873077392578125e-10, &se, &ce);
                            wd = make_double2((double)f * ce, (double)f * se);
                        }
                    }
                }
                if constexpr (EXACT) {
                    if (extra) Ex = cis_exact((uint32_t)(32 * (int)rank + 32) * U, wd);
                }
                float2 R = make_float2(E0.x, E1.x);   // Re of (n, n+1)
                float2 Im = make_float2(E0.y, E1.y);  // Im of (n, n+1)
                if (!wait_bar(&ctl->empty[slot], phase ^ 1u, abort_flag, args.err, args.timeout_ns, 20000u)) {
                    stop = true;
                    break;
                }
                const uint32_t sb = stage_base + (uint32_t)slot * kStageBytes;
                const uint32_t hi_base = is_a ? sb : sb + 2 * kAHalfBytes;
                const uint32_t half_bytes = is_a ? kAHalfBytes : L::kBHalfBytes;
                const uint32_t lo_base = hi_base + half_bytes;
                if (KIND == kTcTile128 && centred) {
                    uint32_t xh = 0u, xl = 0u;  // X(32 rank + 32) as packed (Re, Im)
                    if (extra) split2<BF16>(Ex, xh, xl);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {  // 16 base values
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            if constexpr (EXACT) exact_pair(n0 + 4u * g + 2u * q, U, wd, R, Im);
                            split2<BF16>(R, h[2 * q], l[2 * q]);
                            split2<BF16>(Im, h[2 * q + 1], l[2 * q + 1]);
                            if constexpr (!EXACT) {
                                const float2 Rn = __ffma2_rn(R, ZR, __fmul2_rn(Im, NZI));
                                Im = __ffma2_rn(R, ZI, __fmul2_rn(Im, ZR));
                                R = Rn;
                            }
                        }
                        const uint32_t off = chunk_off(2 * (s0 + 4 * g), k);
                        if (XS_IN_BOUNDS(args.err, slot < kStages && off + 16u <= half_bytes)) {
                            st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
                            st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
                        }
                        if (g == 0 && extra) {
                            // slot 32 takes X(32 rank + 32) in place of X(32 rank)
                            h[0] = __byte_perm(xh, h[0], 0x7610);
                            h[1] = __byte_perm(xh, h[1], 0x7632);
                            l[0] = __byte_perm(xl, l[0], 0x7610);
                            l[1] = __byte_perm(xl, l[1], 0x7632);
                        }
                        const uint32_t moff = chunk_off(2 * (32 + s0 + 4 * g), k);
                        if (XS_IN_BOUNDS(args.err, slot < kStages && moff + 16u <= half_bytes)) {
                            st_shared_v4(hi_base + moff, h[0], h[1], h[2], h[3]);
                            st_shared_v4(lo_base + moff, l[0], l[1], l[2], l[3]);
                        }
                    }
                } else {
#pragma unroll
                    for (int g = 0; g < kRun / 4; ++g) {
                        // one 16-byte chunk = rows (Re n, Re n+1, Im n, Im n+1, Re n+2, Re n+3, Im n+2, Im n+3)
                        uint32_t h[4], l[4];
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            if constexpr (EXACT) exact_pair(n0 + 4u * g + 2u * q, U, wd, R, Im);
                            split2<BF16>(R, h[2 * q], l[2 * q]);
                            split2<BF16>(Im, h[2 * q + 1], l[2 * q + 1]);
                            if constexpr (!EXACT) {
                                const float2 Rn = __ffma2_rn(R, ZR, __fmul2_rn(Im, NZI));
                                Im = __ffma2_rn(R, ZI, __fmul2_rn(Im, ZR));
                                R = Rn;
                            }
                        }
                        const uint32_t off = chunk_off(2 * (run0 + 4 * g), k);
                        if (XS_IN_BOUNDS(args.err, slot < kStages && off + 16u <= half_bytes)) {
                            st_shared_v4(hi_base + off, h[0], h[1], h[2], h[3]);
                            st_shared_v4(lo_base + off, l[0], l[1], l[2], l[3]);
                        }
                    }
                }
                fence_async_shared();
                __syncwarp();
                if (lane == 0) {
                    // CTA-scope release on a barrier of this CTA; in CTA 1 the relay
                    // thread forwards the completed stage to CTA 0 at cluster scope,
                    // once per stage instead of once per producer warp
                    mbar_arrive_local(rank == 0 ? &ctl->full[slot] : &ctl->fill[slot]);
                }
                if (++slot == kStages) {
                    slot = 0;
                    phase ^= 1u;
                }
            }
            up = up_next;
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (rank == 0 && lane == 0) {
            constexpr uint32_t idesc = make_idesc(BF16, 2 * 128, kBN);
            static_assert(kBN % 16 == 0 && kBN >= 16 && kBN <= 256, "MMA N for M = 256");
            int64_t a_cnt = 0;
            int slot = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t ku = 0; ku < my_units && ok; ++ku) {
                const Unit uu = get_unit(args, pair, n_pairs, ku);
                const int n_stages = uu.s1 - uu.s0;
                const int cs = uu.chunk > 0 ? uu.chunk : args.chunk_stages;
                const int n_chunks = (n_stages + cs - 1) / cs;
                for (int c = 0; c < n_chunks && ok; ++c, ++a_cnt) {
                    const int b = (int)(a_cnt & 1);
                    const uint32_t use = (uint32_t)(a_cnt >> 1);
                    if (!wait_bar(&ctl->acc_empty[b], (use & 1u) ^ 1u, abort_flag, args.err, args.timeout_ns,
                                  20000u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)b * (uint32_t)kBN;
                    const int s0 = c * cs;
                    const int s1 = min(n_stages, s0 + cs);
                    for (int s = s0; s < s1; ++s) {
                        if (!wait_bar(&ctl->full[slot], phase, abort_flag, args.err, args.timeout_ns, 20000u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_hi = stage_base + (uint32_t)slot * kStageBytes;
                        const uint32_t a_lo = a_hi + kAHalfBytes;
                        const uint32_t b_hi = a_hi + 2 * kAHalfBytes;
                        const uint32_t b_lo = b_hi + L::kBHalfBytes;
                        if (XS_IN_BOUNDS(args.err, slot < kStages && (uint32_t)(b + 1) * kBN <= C::kTmemCols)) {
#pragma unroll
                            for (int kk = 0; kk < kBK / 16; ++kk) {
                                const uint32_t ko = (uint32_t)kk * 2048u;  // two 8-row K atoms per K = 16
                                umma_pair(d_tmem, mn_desc(a_hi + ko), mn_desc(b_hi + ko), idesc,
                                          (s > s0 || kk > 0) ? 1u : 0u);
                                umma_pair(d_tmem, mn_desc(a_hi + ko), mn_desc(b_lo + ko), idesc, 1u);
                                umma_pair(d_tmem, mn_desc(a_lo + ko), mn_desc(b_hi + ko), idesc, 1u);
                            }
                        }
                        umma_commit_pair(&ctl->empty[slot], 0x3);
                        if (++slot == kStages) {
                            slot = 0;
                            phase ^= 1u;
                        }
                    }
                    if (ok) umma_commit_pair(&ctl->acc_full[b], 0x3);
                }
            }
            // every issued MMA must finish before tensor memory is released
            umma_commit_pair(&ctl->drain, 0x1);
            int no_abort = 0;
            wait_bar(&ctl->drain, 0u, &no_abort, args.err, 2000000000LL, 20000u);
        } else if (rank == 1 && lane == 0) {
            // relay: when this CTA's producers have filled a stage (acquired at
            // CTA scope), arrive on CTA 0's full barrier with a cluster-scope
            // release, which carries their stores to the pair's MMAs
            const uint32_t full_c0 = map_to_rank(smem_u32(&ctl->full[0]), 0);
            int slot = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int64_t ku = 0; ku < my_units && ok; ++ku) {
                const Unit uu = get_unit(args, pair, n_pairs, ku);
                const int n_stages = uu.s1 - uu.s0;
                for (int s = 0; s < n_stages; ++s) {
                    if (!wait_bar(&ctl->fill[slot], phase, abort_flag, args.err, args.timeout_ns, 20000u)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(full_c0 + (uint32_t)slot * 8u);
                    if (++slot == kStages) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        // TMEM lane = A row of this CTA; rows 4g..4g+3 are (Re x, Re x+1, Im x, Im x+1)
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const int row = warp * 32 + lane;
        const bool re_row = (lane & 2) == 0;
        const int x_slot = 2 * (row >> 2) + (row & 1);
        float sx_c;
        const int xi_c = centred_index(x_slot, (int)rank, sx_c);
        float2* scr = reinterpret_cast<float2*>(args.scratch) + (size_t)blockIdx.x * 256 * 128 + row;
        const uint32_t acc_empty_c0 = map_to_rank(smem_u32(&ctl->acc_empty[0]), 0);
        int64_t a_cnt = 0;
        bool ok = true;
        for (int64_t ku = 0; ku < my_units && ok; ++ku) {
            const Unit up = get_unit(args, pair, n_pairs, ku);
            const int cs = up.chunk > 0 ? up.chunk : args.chunk_stages;
            const int n_chunks = (up.s1 - up.s0 + cs - 1) / cs;
            const bool centred = KIND == kTcTile128 && up.centred;
            // narrow tiles: rows x_slot < kHalf / 2 hold n_x (kHalf / 2) rank +
            // x_slot, the others were not built (-1: nothing written)
            const int xi = centred ? xi_c
                                   : (unit_narrow(up, centred) ? (x_slot < kHalf / 2 ? (kHalf / 2) * (int)rank + x_slot : -1)
                                                               : kHalf * (int)rank + x_slot);
            const double sx = centred ? (double)sx_c : 1.0;  // sign of the stored Im x rows
            for (int c = 0; c < n_chunks; ++c, ++a_cnt) {
                const int b = (int)(a_cnt & 1);
                const uint32_t use = (uint32_t)(a_cnt >> 1);
                uint32_t got = 0;
                if (lane == 0)
                    got = wait_bar(&ctl->acc_full[b], use & 1u, abort_flag, args.err, args.timeout_ns, 200000u);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dcol = lane_base + (uint32_t)b * (uint32_t)kBN;
                const bool first = c == 0, last = c == n_chunks - 1;
#pragma unroll 1
                for (int j = 0; j < kBN / 16; ++j) {
                    uint32_t r[16];
                    if (XS_IN_BOUNDS(args.err, row < 128 && (uint32_t)b * kBN + 16u * (j + 1) <= C::kTmemCols)) {
                        tmem_ld16(dcol + 16 * j, r);
                        tmem_wait16(r);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) r[i] = 0u;
                    }
                    // scratch rows of this thread for columns 16j .. 16j+15
                    const bool scr_ok = XS_IN_BOUNDS(
                        args.err, (int64_t)blockIdx.x * 256 * 128 + row + (int64_t)(16 * j + 15) * 128 < args.scratch_f2);
                    // running total per value as an unevaluated FP32 pair hi + lo,
                    // updated with the error-free sum TwoSum(hi, chunk)
                    float hi[16], lo[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float c = __uint_as_float(r[i]);
                        if (first || !scr_ok) {
                            hi[i] = c;
                            lo[i] = 0.0f;
                        } else {
                            const float2 t = scr[(size_t)(16 * j + i) * 128];
                            const float s = t.x + c;
                            const float bb = s - t.x;
                            const float e = (t.x - (s - bb)) + (c - bb);
                            hi[i] = s;
                            lo[i] = t.y + e;
                        }
                    }
                    if (!last) {
                        if (scr_ok) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) scr[(size_t)(16 * j + i) * 128] = make_float2(hi[i], lo[i]);
                        }
                        continue;
                    }
                    double v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = (double)hi[i] + (double)lo[i];
                    // columns 16j .. 16j+15 hold n_y local m = 8j .. 8j+7 in groups of 4
                    // (Re m, Re m+1, Im m, Im m+1): CTA r's B rows are columns
                    // [r kBN / 2, (r + 1) kBN / 2), n_y [r kTileY / 2, ...), so
                    // m = 8j for both tile kinds; the Re lane finishes m = 8j..8j+3 with
                    // the Im values of its partner lane (lane ^ 2), the Im lane m = 8j+4..8j+7
                    double own[8], rcv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        own[i] = re_row ? v[i] : v[8 + i];
                        const double snd = re_row ? v[8 + i] : v[i];
                        rcv[i] = __shfl_xor_sync(0xffffffffu, snd, 2);
                    }
                    const int ix = up.tx * kTile + xi;
                    // a piece of a split unit keeps its partial amplitude of every pixel
                    double2* part_dst = up.split >= 0 && xi >= 0
                                            ? args.partial +
                                                  ((size_t)up.split * args.parts + up.part) * (kTile * kTile) +
                                                  (size_t)xi * kTile
                                            : nullptr;
                    if (xi >= 0 && (part_dst || ix < up.nx)) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const double* vr = re_row ? own : rcv;  // D[Re x][...]
                                const double* vi = re_row ? rcv : own;  // D[Im x][...]
                                const double p_rr = vr[4 * hh + t], p_ri = vr[4 * hh + 2 + t];
                                const double p_ir = vi[4 * hh + t], p_ii = vi[4 * hh + 2 + t];
                                const int m = 8 * j + (re_row ? 0 : 4) + 2 * hh + t;
                                int yi = m;
                                double sy = 1.0;  // sign of the stored Im y rows
                                if (centred) {
                                    float f;
                                    yi = centred_index(m & (kHalf - 1), m / kHalf, f);
                                    sy = (double)f;
                                }
                                const double sre = p_rr - sx * sy * p_ii;
                                const double sim = sy * p_ri + sx * p_ir;
                                const int iy = up.ty * C::kTileY + yi;
                                if (part_dst) {
                                    if (XS_IN_BOUNDS(args.err, ((int64_t)up.split * args.parts + up.part) * (kTile * kTile) +
                                                                       (int64_t)xi * kTile + yi <
                                                                   args.partial_n))
                                        part_dst[yi] = make_double2(sre, sim);
                                } else if (iy < up.ny) {
                                    const int64_t o = (((int64_t)up.t * up.nz + up.iz) * up.ny + iy) * up.nx + ix;
                                    if (XS_IN_BOUNDS(args.err, o >= 0 && o < up.out_n)) {
                                        up.I[o] = (float)(sre * sre + sim * sim);
                                        if (up.amp) {
                                            up.amp[2 * o] = (float)sre;
                                            up.amp[2 * o + 1] = (float)sim;
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acc_empty_c0 + (uint32_t)b * 8u);
            }
        }
    }

    __syncwarp();
    tc_fence_before();
    cluster_sync();  // no CTA leaves while the pair's MMAs or its peer may still touch it
    tc_fence_after();
    if (warp == 0) tmem_dealloc_pair(tmem, C::kTmemCols);
}

}  // namespace

bool tc_supported(const GridDesc& g) { return g.nx >= 1 && g.ny >= 1 && g.nz >= 1; }

int64_t tc_atom_multiple() { return kBK; }

template <int KIND>
static int pair_capacity_of(int num_sms) {
    // pairs that can be resident at once (a cluster needs two SMs of one GPC)
    static int max_pairs = -1;
    if (max_pairs < 0) {
        using L = Lay<KIND>;
        cudaFuncSetAttribute((const void*)tc_kernel<false, KIND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L::kSmemBytes);
        cudaFuncSetAttribute((const void*)tc_kernel<true, KIND, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)L::kSmemBytes);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (unsigned)std::max(1, num_sms / 2), 1, 1);
        cfg.blockDim = dim3(L::kThreads, 1, 1);
        cfg.dynamicSmemBytes = L::kSmemBytes;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 2;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (const void*)tc_kernel<false, KIND, false>, &cfg) != cudaSuccess ||
            n < 1) {
            cudaGetLastError();
            n = std::max(1, num_sms / 2);
        }
        max_pairs = n;
    }
    return max_pairs;
}

int tc_pair_capacity(int num_sms, int kind) {
    return kind == kTcTile64 ? pair_capacity_of<kTcTile64>(num_sms) : pair_capacity_of<kTcTile128>(num_sms);
}

int tc_default_kind(const GridDesc& g) { return g.ny <= 64 ? kTcTile64 : kTcTile128; }

#ifdef XS_BOUNDS_CHECK
// Self-test of the checked build: with XS_CHECK_SHORT_OUTPUT=1 the bounds
// check of tc_kernel admits one frame of I less than the buffers hold, so the
// last frame's writes fail the check and are skipped (every access stays
// inside the real buffers) and the call returns XS_ERR_BOUNDS.
static bool check_short_output() {
    static const bool on = [] {
        const char* v = std::getenv("XS_CHECK_SHORT_OUTPUT");
        return v && v[0] == '1';
    }();
    return on;
}
#endif

TcTraj tc_traj(const AtomRec* rec, int64_t n_pad, int64_t n_frames, const GridDesc& g, float* I, float* amp, int kind,
               int chunk, bool exact) {
    TcTraj t;
    t.exact = exact ? 1 : 0;
    t.kind = kind == kTcTile64 ? kTcTile64 : kTcTile128;
    t.chunk = chunk;
    t.rec = reinterpret_cast<const uint4*>(rec);
    t.I = I;
    t.amp = amp;
    t.n_pad = n_pad;
    t.n_stages = (int)(n_pad / kBK);
    t.tiles_x = (g.nx + kTile - 1) / kTile;
    t.tiles_y = (g.ny + tc_tile_y(t.kind) - 1) / tc_tile_y(t.kind);
    t.nx0 = g.nx0;
    t.nx = g.nx;
    t.ny0 = g.ny0;
    t.ny = g.ny;
    t.nz0 = g.nz0;
    t.nz = g.nz;
    t.n_frames = (int)n_frames;
#ifdef XS_BOUNDS_CHECK
    t.check_frames = (int)n_frames - (check_short_output() ? 1 : 0);
#endif
    return t;
}

int64_t tc_units(const TcTraj& t) { return (int64_t)t.n_frames * t.nz * t.tiles_x * t.tiles_y; }

size_t tc_scratch_bytes(int n_pairs) { return (size_t)(2 * n_pairs) * 256 * 128 * sizeof(double); }

void tc_build_lists(const std::vector<TcTraj>& trajs, int n_pairs, std::vector<int4>& units,
                    std::vector<int>& pair_start) {
    std::vector<int4> all;
    for (size_t i = 0; i < trajs.size(); ++i) {
        const TcTraj& t = trajs[i];
        for (int f = 0; f < t.n_frames; ++f)
            for (int z = 0; z < t.nz; ++z)
                for (int ty = 0; ty < t.tiles_y; ++ty)
                    for (int tx = 0; tx < t.tiles_x; ++tx) all.push_back(make_int4((int)i, f, z, tx | (ty << 16)));
    }
    tc_deal_units(trajs, all, n_pairs, units, pair_start);
}

void tc_deal_units(const std::vector<TcTraj>& trajs, const std::vector<int4>& all, int n_pairs,
                   std::vector<int4>& units, std::vector<int>& pair_start) {
    // longest-processing-time first: units sorted by cost (stages), each given
    // to the least loaded pair; ties keep the given order
    struct Item {
        int64_t cost;
        int4 u;
    };
    std::vector<Item> items;
    items.reserve(all.size());
    for (const int4& u : all) items.push_back({trajs[(size_t)u.x].n_stages, u});
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.cost > b.cost; });
    using Load = std::pair<int64_t, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int p = 0; p < n_pairs; ++p) heap.push({0, p});
    std::vector<std::vector<int4>> per(n_pairs);
    for (const Item& it : items) {
        Load l = heap.top();
        heap.pop();
        per[l.second].push_back(it.u);
        heap.push({l.first + it.cost, l.second});
    }
    units.clear();
    pair_start.assign((size_t)n_pairs + 1, 0);
    for (int p = 0; p < n_pairs; ++p) {
        pair_start[p] = (int)units.size();
        units.insert(units.end(), per[p].begin(), per[p].end());
    }
    pair_start[n_pairs] = (int)units.size();
}

template <bool BF16, int KIND, bool EXACT>
static cudaError_t launch_kind(const TcArgs& a, int n_pairs, cudaStream_t st) {
    using L = Lay<KIND>;
    const void* fn = (const void*)tc_kernel<BF16, KIND, EXACT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::kSmemBytes);
    if (e != cudaSuccess) return e;
    ++tl_kernel_launches;
    tc_kernel<BF16, KIND, EXACT><<<2 * n_pairs, L::kThreads, L::kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

template <bool EXACT>
static cudaError_t launch_exact(const TcArgs& a, int n_pairs, bool bf16, int kind, cudaStream_t st) {
    if (kind == kTcTile64)
        return bf16 ? launch_kind<true, kTcTile64, EXACT>(a, n_pairs, st)
                    : launch_kind<false, kTcTile64, EXACT>(a, n_pairs, st);
    return bf16 ? launch_kind<true, kTcTile128, EXACT>(a, n_pairs, st)
                : launch_kind<false, kTcTile128, EXACT>(a, n_pairs, st);
}

static cudaError_t launch(const TcArgs& a, int n_pairs, bool bf16, int kind, bool exact, cudaStream_t st) {
    return exact ? launch_exact<true>(a, n_pairs, bf16, kind, st) : launch_exact<false>(a, n_pairs, bf16, kind, st);
}

TcSplit tc_split_plan(int64_t units, int n_pairs, int n_stages, int chunk_stages) {
    // Units are dealt round-robin; when the last wave is partial, its units
    // are cut along the atoms into `parts` pieces so that the last wave takes
    // ceil(rem * parts / n_pairs) / parts of a unit instead of a whole one.
    constexpr int kMaxParts = 16;
    constexpr int64_t kMaxPieces = 1024;  // 256 KB of partial amplitudes each
    TcSplit sp;
    sp.full = 0;
    sp.rem = units;
    sp.parts = 1;
    if (units <= 0 || n_pairs <= 0) return sp;
    const int64_t F = units / n_pairs, R = units % n_pairs;
    if (R == 0) return sp;
    const int chunk = chunk_stages > 0 ? chunk_stages : 32;
    int best = 1;
    double best_cost = 1.0;
    for (int k = 2; k <= kMaxParts; ++k) {
        if (n_stages / k < 2 * chunk || R * k > kMaxPieces) break;  // pieces of two chunks at least
        const double cost = (double)((R * k + n_pairs - 1) / n_pairs) / k;
        if (cost < best_cost - 1e-9) {
            best = k;
            best_cost = cost;
        }
    }
    if (best == 1) return sp;
    sp.full = F;
    sp.rem = R;
    sp.parts = best;
    return sp;
}

size_t tc_split_bytes(const TcSplit& sp) {
    if (sp.parts <= 1) return 0;
    return (size_t)sp.rem * sp.parts * kTile * kTile * sizeof(double2);
}

cudaError_t launch_tc_single(const TcTraj& tr, int n_pairs, const TcSplit& sp, int chunk_stages, bool bf16,
                             double* scratch, void* split_buf, int* err, int64_t timeout_ns, cudaStream_t st) {
    if (tr.n_pad % kBK != 0) return cudaErrorInvalidValue;
    const int64_t units = tc_units(tr);
    if (units == 0) return cudaSuccess;
    if (sp.full * n_pairs + sp.rem != units || sp.parts < 1) return cudaErrorInvalidValue;
    TcArgs a{};
    a.single = tr;
    a.full = sp.full;
    a.rem = sp.rem;
    a.parts = sp.parts;
    a.chunk_stages = chunk_stages > 0 ? chunk_stages : 32;
    a.scratch = scratch;
    a.err = err;
    a.timeout_ns = timeout_ns;
    if (sp.parts > 1) {
        if (!split_buf) return cudaErrorInvalidValue;
        a.partial = static_cast<double2*>(split_buf);
    }
#ifdef XS_BOUNDS_CHECK
    a.scratch_f2 = (int64_t)(tc_scratch_bytes(n_pairs) / sizeof(float2));
    a.partial_n = (int64_t)(tc_split_bytes(sp) / sizeof(double2));
#endif
    const int64_t pieces = sp.full * n_pairs + sp.rem * sp.parts;
    n_pairs = (int)std::min<int64_t>(n_pairs, pieces);
    return launch(a, n_pairs, bf16, tr.kind, tr.exact != 0, st);
}

cudaError_t launch_tc_split_finish(const TcTraj& tr, int n_pairs, const TcSplit& sp, void* split_buf,
                                   cudaStream_t st) {
    if (sp.parts <= 1 || sp.rem == 0) return cudaSuccess;
    if (!split_buf) return cudaErrorInvalidValue;
    TcArgs a{};
    a.single = tr;
    a.full = sp.full;
    a.rem = sp.rem;
    a.parts = sp.parts;
    a.partial = static_cast<double2*>(split_buf);
    const int64_t pieces = sp.full * n_pairs + sp.rem * sp.parts;
    n_pairs = (int)std::min<int64_t>(n_pairs, pieces);  // as in launch_tc_single
    ++tl_kernel_launches;
    split_finish_kernel<<<dim3(kTile * kTile / 256, (unsigned)sp.rem), 256, 0, st>>>(a, n_pairs);
    return cudaGetLastError();
}

cudaError_t launch_tc_batch(const TcTraj* d_trajs, const int4* d_units, const int* d_pair_start, int n_pairs,
                            int chunk_stages, bool bf16, int kind, bool exact, double* scratch, int* err,
                            int64_t timeout_ns, cudaStream_t st) {
    TcArgs a{};
    a.trajs = d_trajs;
    a.units = d_units;
    a.pair_start = d_pair_start;
    a.chunk_stages = chunk_stages > 0 ? chunk_stages : 32;
    a.scratch = scratch;
    a.err = err;
    a.timeout_ns = timeout_ns;
#ifdef XS_BOUNDS_CHECK
    a.scratch_f2 = (int64_t)(tc_scratch_bytes(n_pairs) / sizeof(float2));
#endif
    return launch(a, n_pairs, bf16, kind, exact, st);
}

}  // namespace xs
