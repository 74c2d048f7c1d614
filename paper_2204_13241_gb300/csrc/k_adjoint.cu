// Adjoint of the intensity with respect to atomic positions.
//
//   dL/dr_j = sum_q G_q 2 Re[conj(S_q) i q f_j e^{i q.r_j}]
//           = -2 f_j sum_q Im[H_q e^{i theta_qj}] q,          H_q = G_q conj(S_q)
// With q = 2 pi h^-T n and theta = 2 pi (n_x s_x + n_y s_y + n_z s_z):
//   dL/dr_j = -4 pi f_j h^-T Im[T_j],   T_j,a = sum_q n_a H_q e^{i theta_qj}.
// Because the phase factorises over the axes (Sec. 3.1, reciprocal-lattice q),
//   T_x = sum_{z,x} n_x E_xz Z,  T_y = sum_{z,x} E_xz Z_y,  T_z = sum_{z,x} n_z E_xz Z
// with Z(x,z) = sum_y H(x,y,z) E_y and Z_y(x,z) = sum_y n_y H(x,y,z) E_y:
// two complex contractions over n_y followed by per-atom sums over n_x, n_z.
//
// adjoint_kernel: a block owns 64 atoms.  The factors E_y[n_y][atom] of a
// chunk of up to 256 n_y rows are built in shared memory from exact integer
// phases; each warp owns every 8th n_x row and each lane two atoms; H rows are
// read warp-uniformly from global memory (L1/L2 resident).  Partial T of the 8
// warps are added in a fixed order.  All arithmetic is FP32 except the final
// scaling.
#include "xs_internal.h"

namespace xs {

namespace {

constexpr bool kAdjointOnTensorCores = true;  // false: the FP32 kernel below
constexpr int kAdjAtoms = 64;
constexpr int kAdjThreads = 256;
constexpr int kAdjWarps = kAdjThreads / 32;
constexpr int kAdjYChunk = 128;  // n_y rows of E_y per shared-memory chunk (64 KB: three blocks per SM)

__global__ void h_kernel(const float* __restrict__ amp, const float* __restrict__ G, int64_t P,
                         float2* __restrict__ H) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[p];
        H[p] = make_float2(g * amp[2 * p], -g * amp[2 * p + 1]);
    }
}

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

__global__ void __launch_bounds__(kAdjThreads, 1)
adjoint_kernel(const AtomRec* __restrict__ rec, int64_t n_atoms, GridDesc g, Mat3 hinv,
               const float2* __restrict__ H, float* __restrict__ grad) {
    extern __shared__ float2 s_ey[];  // [kAdjYChunk][kAdjAtoms]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile0 = (int64_t)blockIdx.x * kAdjAtoms;
    const int la[2] = {lane, lane + 32};
    AtomRec ar[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) ar[k] = rec[tile0 + la[k]];

    float2 Tx[2], Ty[2], Tz[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) Tx[k] = Ty[k] = Tz[k] = make_float2(0.f, 0.f);

    const int64_t plane = (int64_t)g.nx * g.ny;
    for (int cy0 = 0; cy0 < g.ny; cy0 += kAdjYChunk) {
        const int ncy = min(kAdjYChunk, g.ny - cy0);
        __syncthreads();
        for (int e = threadIdx.x; e < ncy * kAdjAtoms; e += kAdjThreads) {
            const int iy = e / kAdjAtoms, a = e - iy * kAdjAtoms;
            const uint32_t ny = (uint32_t)(g.ny0 + cy0 + iy);
            float c, s;
            phase_to_cs(ny * rec[tile0 + a].uy, c, s);
            s_ey[e] = make_float2(c, s);
        }
        __syncthreads();
        for (int iz = 0; iz < g.nz; ++iz) {
            const uint32_t nz = (uint32_t)(g.nz0 + iz);
            const float fnz = (float)(g.nz0 + iz);
            for (int ix0 = warp; ix0 < g.nx; ix0 += 2 * kAdjWarps) {
                const int ix1 = ix0 + kAdjWarps;
                const bool has1 = ix1 < g.nx;
                const float2* h0 = H + iz * plane + (int64_t)cy0 * g.nx + ix0;
                const float2* h1 = H + iz * plane + (int64_t)cy0 * g.nx + (has1 ? ix1 : ix0);
                float2 Z[2][2], Zy[2][2];
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int k = 0; k < 2; ++k) Z[r][k] = Zy[r][k] = make_float2(0.f, 0.f);
                float fny = (float)(g.ny0 + cy0);
                // h1 aliases h0 when the warp has no second row; its sums are
                // then never used.  Pointer steps, no index products.
#pragma unroll 2
                for (int iy = 0; iy < ncy; ++iy, fny += 1.0f, h0 += g.nx, h1 += g.nx) {
                    const float2 hv0 = *h0;
                    const float2 hv1 = *h1;
                    const float2 hy0 = make_float2(fny * hv0.x, fny * hv0.y);
                    const float2 hy1 = make_float2(fny * hv1.x, fny * hv1.y);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const float2 e = s_ey[iy * kAdjAtoms + la[k]];
                        cmac(Z[0][k], hv0, e);
                        cmac(Zy[0][k], hy0, e);
                        cmac(Z[1][k], hv1, e);
                        cmac(Zy[1][k], hy1, e);
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if (r == 1 && !has1) break;
                    const int ix = r == 0 ? ix0 : ix1;
                    const uint32_t nx = (uint32_t)(g.nx0 + ix);
                    const float fnx = (float)(g.nx0 + ix);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        float c, s;
                        phase_to_cs(nx * ar[k].ux + nz * ar[k].uz, c, s);
                        const float2 E = make_float2(c, s);
                        float2 ez = make_float2(0.f, 0.f), ezy = make_float2(0.f, 0.f);
                        cmac(ez, E, Z[r][k]);
                        cmac(ezy, E, Zy[r][k]);
                        Tx[k].x = fmaf(fnx, ez.x, Tx[k].x);
                        Tx[k].y = fmaf(fnx, ez.y, Tx[k].y);
                        Ty[k].x += ezy.x;
                        Ty[k].y += ezy.y;
                        Tz[k].x = fmaf(fnz, ez.x, Tz[k].x);
                        Tz[k].y = fmaf(fnz, ez.y, Tz[k].y);
                    }
                }
            }
        }
    }
    // fixed-order sum of the warps' partial Im[T]
    __syncthreads();
    float* red = reinterpret_cast<float*>(s_ey);  // [warp][atom][3]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float* o = red + (warp * kAdjAtoms + la[k]) * 3;
        o[0] = Tx[k].y;
        o[1] = Ty[k].y;
        o[2] = Tz[k].y;
    }
    __syncthreads();
    if (threadIdx.x < kAdjAtoms) {
        const int a = threadIdx.x;
        const int64_t j = tile0 + a;
        if (j < n_atoms) {
            double v[3] = {0.0, 0.0, 0.0};
            for (int w = 0; w < kAdjWarps; ++w)
                for (int c = 0; c < 3; ++c) v[c] += (double)red[(w * kAdjAtoms + a) * 3 + c];
            const double scale = -4.0 * 3.14159265358979323846 * (double)rec[j].f;
            // (h^-T v)_a = sum_b hinv[b][a] v_b
            for (int c = 0; c < 3; ++c) {
                const double hv = hinv.a[0 * 3 + c] * v[0] + hinv.a[1 * 3 + c] * v[1] + hinv.a[2 * 3 + c] * v[2];
                grad[j * 3 + c] = (float)(scale * hv);
            }
        }
    }
}

}  // namespace

static size_t h_bytes(const GridDesc& g) { return ((size_t)g.pixels() * sizeof(float2) + 1023) & ~(size_t)1023; }

size_t adjoint_workspace_bytes(const GridDesc& g) { return h_bytes(g) + adjoint_tc_image_bytes(g); }

cudaError_t launch_adjoint(const AtomRec* rec, int64_t n_atoms, int64_t n_pad, const GridDesc& g,
                           const Mat3& hinv, const float* amp, const float* dL_dI, void* workspace,
                           float* grad, int* err, int64_t timeout_ns, cudaStream_t st) {
    const int64_t P = g.pixels();
    float2* H = static_cast<float2*>(workspace);
    const int64_t hb = min((P + 255) / 256, (int64_t)4096);
    ++tl_kernel_launches;
    h_kernel<<<(unsigned)hb, 256, 0, st>>>(amp, dL_dI, P, H);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (kAdjointOnTensorCores)
        return launch_adjoint_tc(rec, n_atoms, n_pad, g, hinv, H, static_cast<char*>(workspace) + h_bytes(g), grad,
                                 err, timeout_ns, st);
    const size_t smem = (size_t)kAdjYChunk * kAdjAtoms * sizeof(float2);
    e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = n_pad / kAdjAtoms;
    ++tl_kernel_launches;
    adjoint_kernel<<<(unsigned)blocks, kAdjThreads, smem, st>>>(rec, n_atoms, g, hinv, H, grad);
    return cudaGetLastError();
}

}  // namespace xs
