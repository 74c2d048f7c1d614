// Several atom species with q-dependent form factors (Sec. 2.1: f_i(q), each
// species' form factor a sum of Gaussians in |q|).  The amplitude splits by
// species, S(q) = sum_s F_s(q) S_s(q) with S_s the plain direct sum over the
// atoms of species s (per-atom weights kept), so each species runs through the
// same phase and contraction kernels and these kernels combine the results:
//   ff_table_kernel      F_s(|q_p|) for every species and pixel, FP64
//   species_acc_kernel   acc[t][p] (+)= F_s(q_p) S_s[t][p], FP64 complex
//   species_finish_kernel I = |acc|^2 and the amplitude, FP32
// and the gather of arbitrary lattice points out of the planes that hold them
// (points_gather_kernel), and the fill of a grid from the half of it that the
// contraction computed (friedel_kernel: for real form factors S(-q) =
// conj S(q), so I(-q) = I(q), as the pair form of the intensity, a sum of
// f_i f_j cos(q.r_ij), shows).
#include <algorithm>
#include <cmath>

#include "xs_internal.h"

namespace xs {

namespace {

// one thread per pixel: |q| = |2 pi h^-T n|, s = |q| / (4 pi),
// F = sum_k a_k exp(-b_k s^2) + c for every species
__global__ void ff_table_kernel(const double* __restrict__ coef, int n_species, GridDesc g, Mat3 hinv,
                                double* __restrict__ table) {
    const int64_t P = g.pixels();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int iz = (int)(p / plane);
    const int64_t rem = p - (int64_t)iz * plane;
    const int iy = (int)(rem / g.nx);
    const int ix = (int)(rem - (int64_t)iy * g.nx);
    const double n[3] = {(double)(g.nx0 + ix), (double)(g.ny0 + iy), (double)(g.nz0 + iz)};
    double q2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        // q_a = 2 pi sum_b (h^-1)_{b a} n_b
        const double qa = 6.283185307179586 * (hinv.a[0 * 3 + a] * n[0] + hinv.a[1 * 3 + a] * n[1] +
                                               hinv.a[2 * 3 + a] * n[2]);
        q2 += qa * qa;
    }
    const double s2 = q2 / (16.0 * 9.869604401089358);  // |q|^2 / (4 pi)^2
    for (int sp = 0; sp < n_species; ++sp) {
        const double* c = coef + 9 * sp;
        double v = c[8];
        for (int k = 0; k < 4; ++k) v += c[2 * k] * exp(-c[2 * k + 1] * s2);
        table[(int64_t)sp * P + p] = v;
    }
}

__global__ void species_acc_kernel(const float2* __restrict__ S, const double* __restrict__ ff, int64_t nf,
                                   int64_t P, bool first, double2* __restrict__ acc) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nf * P) return;
    const double w = ff[i % P];
    const float2 z = S[i];
    double2 a = first ? make_double2(0.0, 0.0) : acc[i];
    a.x = fma(w, (double)z.x, a.x);
    a.y = fma(w, (double)z.y, a.y);
    acc[i] = a;
}

__global__ void species_finish_kernel(const double2* __restrict__ acc, int64_t n, float* __restrict__ I,
                                      float* __restrict__ amp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 a = acc[i];
    I[i] = (float)(a.x * a.x + a.y * a.y);
    if (amp) {
        amp[2 * i] = (float)a.x;
        amp[2 * i + 1] = (float)a.y;
    }
}

// out[t][p] = tmp[src[p] + t * stride[p]] (and the amplitude), one thread per (t, p)
__global__ void points_gather_kernel(const float* __restrict__ tmp, const float* __restrict__ tmp_amp,
                                     const int64_t* __restrict__ src, const int64_t* __restrict__ stride,
                                     int64_t P, int64_t nf, float* __restrict__ I, float* __restrict__ amp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nf * P) return;
    const int64_t t = i / P, p = i - t * P;
    const int64_t o = src[p] + t * stride[p];
    I[i] = tmp[o];
    if (amp) {
        amp[2 * i] = tmp_amp[2 * o];
        amp[2 * i + 1] = tmp_amp[2 * o + 1];
    }
}

// one thread per output pixel of I [T][nz][ny][nx] (grid g): pixels whose
// coordinate on the split axis is <= 0 are read from the half-grid `half`
// [T][v.nz][v.ny][v.nx], the others from their mirror -n (the amplitude is
// conjugated there)
__global__ void friedel_kernel(const float* __restrict__ half, const float* __restrict__ half_amp, int64_t T,
                               GridDesc v, GridDesc g, int axis, float* __restrict__ I, float* __restrict__ amp) {
    const int64_t P = g.pixels();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T * P) return;
    const int64_t t = i / P;
    const int64_t p = i - t * P;
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int iz = (int)(p / plane);
    const int64_t rem = p - (int64_t)iz * plane;
    const int iy = (int)(rem / g.nx);
    const int ix = (int)(rem - (int64_t)iy * g.nx);
    int n[3] = {g.nx0 + ix, g.ny0 + iy, g.nz0 + iz};
    const bool mirror = n[axis] > 0;
    if (mirror) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
    }
    const int64_t o = ((t * v.nz + (n[2] - v.nz0)) * v.ny + (n[1] - v.ny0)) * v.nx + (n[0] - v.nx0);
    I[i] = half[o];
    if (amp) {
        amp[2 * i] = half_amp[2 * o];
        amp[2 * i + 1] = mirror ? -half_amp[2 * o + 1] : half_amp[2 * o + 1];
    }
}

}  // namespace

int friedel_half_grid(const GridDesc& g, GridDesc& v) {
    // For real form factors I(-n) = I(n): the pixels of g whose coordinate on
    // the split axis (n_x for a plane at n_z = 0, n_z otherwise) is positive
    // are read from their mirrors.  The half-grid v keeps the split axis from
    // min(lo, 1 - hi) to 0 and widens the other two to the hull of their
    // range and its mirror.  It is used where it needs fewer 128 x 128 tiles
    // (planes of 192^2: 2 instead of 4; the volume n in [-40, 40]^3: 41
    // instead of 81).
    const int axis = (g.nz == 1 && g.nz0 == 0) ? 0 : 2;
    int lo[3] = {g.nx0, g.ny0, g.nz0}, n[3] = {g.nx, g.ny, g.nz};
    int vlo[3], vn[3];
    for (int a = 0; a < 3; ++a) {
        const int hi = lo[a] + n[a];  // exclusive
        if (a == axis) {
            if (hi <= 1) return -1;  // nothing positive to mirror
            vlo[a] = std::min(lo[a], 1 - hi);
            vn[a] = 1 - vlo[a];      // up to 0 inclusive
        } else {
            vlo[a] = std::min(lo[a], 1 - hi);
            vn[a] = std::max(hi, 1 - lo[a]) - vlo[a];
        }
    }
    v = g;
    v.nx0 = vlo[0];
    v.nx = vn[0];
    v.ny0 = vlo[1];
    v.ny = vn[1];
    v.nz0 = vlo[2];
    v.nz = vn[2];
    auto tiles = [](const GridDesc& d) { return (int64_t)d.nz * ((d.nx + 127) / 128) * ((d.ny + 127) / 128); };
    return tiles(v) < tiles(g) ? axis : -1;
}

cudaError_t launch_friedel(const float* half, const float* half_amp, int64_t T, const GridDesc& v, const GridDesc& g,
                           int axis, float* I, float* amp, cudaStream_t st) {
    const int64_t n = T * g.pixels();
    if (n == 0) return cudaSuccess;
    ++tl_kernel_launches;
    friedel_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(half, half_amp, T, v, g, axis, I, amp);
    return cudaGetLastError();
}

cudaError_t launch_points_gather(const float* tmp, const float* tmp_amp, const int64_t* d_src, const int64_t* d_stride,
                                 int64_t P, int64_t nf, float* I, float* amp, cudaStream_t st) {
    const int64_t n = nf * P;
    if (n == 0) return cudaSuccess;
    ++tl_kernel_launches;
    points_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmp, tmp_amp, d_src, d_stride, P, nf, I, amp);
    return cudaGetLastError();
}

cudaError_t launch_ff_table(const double* d_coef, int n_species, const GridDesc& g, const Mat3& hinv, double* table,
                            cudaStream_t st) {
    const int64_t P = g.pixels();
    if (P == 0 || n_species == 0) return cudaSuccess;
    ++tl_kernel_launches;
    ff_table_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(d_coef, n_species, g, hinv, table);
    return cudaGetLastError();
}

cudaError_t launch_species_acc(const float* S, const double* ff, int64_t nf, int64_t P, bool first, double* acc,
                               cudaStream_t st) {
    const int64_t n = nf * P;
    if (n == 0) return cudaSuccess;
    ++tl_kernel_launches;
    species_acc_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float2*>(S), ff, nf, P,
                                                                    first, reinterpret_cast<double2*>(acc));
    return cudaGetLastError();
}

cudaError_t launch_species_finish(const double* acc, int64_t n, float* I, float* amp, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    ++tl_kernel_launches;
    species_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const double2*>(acc), n, I,
                                                                       amp);
    return cudaGetLastError();
}

}  // namespace xs
