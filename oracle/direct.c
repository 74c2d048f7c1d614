/*
 * FP64 CPU oracle for the direct method -- TEST INFRASTRUCTURE ONLY.
 *
 * Nothing on the product path may call this file.  It is a plain, slow,
 * obviously correct restatement of the paper's definitions, used by the
 * tests, by the bench's CPU-baseline leg and by the smoke check.
 *
 * Definitions followed (arXiv 2204.13241):
 *   Sec. 2.2, Eq. pe_ri : p^e(q,t) = sum_i f_i exp(-i q.r_i(t)).
 *   Sec. 2.2, Eq. Iq_pq : I(q,t) = |p^e(q,t)|^2.
 *   Sec. 3.1, Eq. sq_cut_simple and Algorithm 1 : evaluate the single sum
 *     over atoms at each q of a grid on the reciprocal lattice of the box,
 *     q = 2 pi h^-T n  (for a cubic box of side L, q = 2 pi n / L).
 * Sign convention of this library: S(q) = sum_j f_j exp(+i q.r_j), the
 * complex conjugate of the paper's p^e; I = |S|^2 is identical.
 *
 * Arithmetic: the phase q.r is formed in FP64 from the float32 positions
 * promoted to double, sin/cos are libm's, and the real and imaginary sums use
 * Neumaier compensated summation.  The cell matrix h (row-major, columns are
 * the cell edge vectors) is inverted here with the cofactor formula.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double s, c; } neumaier;

static inline void nm_add(neumaier* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static inline double nm_value(const neumaier* a) { return a->s + a->c; }

/* inverse of a 3x3 row-major matrix by cofactors; returns 0 when singular */
int oracle_inverse3(const double* h, double* hinv) {
    double c00 = h[4] * h[8] - h[5] * h[7];
    double c01 = h[5] * h[6] - h[3] * h[8];
    double c02 = h[3] * h[7] - h[4] * h[6];
    double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (det == 0.0 || !isfinite(det)) return 0;
    double id = 1.0 / det;
    hinv[0] = c00 * id;
    hinv[1] = (h[2] * h[7] - h[1] * h[8]) * id;
    hinv[2] = (h[1] * h[5] - h[2] * h[4]) * id;
    hinv[3] = c01 * id;
    hinv[4] = (h[0] * h[8] - h[2] * h[6]) * id;
    hinv[5] = (h[2] * h[3] - h[0] * h[5]) * id;
    hinv[6] = c02 * id;
    hinv[7] = (h[1] * h[6] - h[0] * h[7]) * id;
    hinv[8] = (h[0] * h[4] - h[1] * h[3]) * id;
    return 1;
}

/* q = 2 pi h^-T n  for every Miller index; q_out [n_q][3] */
int oracle_qvectors(const double* h, const int32_t* miller, int64_t n_q, double* q_out) {
    double hi[9];
    if (!oracle_inverse3(h, hi)) return 0;
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t p = 0; p < n_q; ++p) {
        double n0 = miller[3 * p + 0], n1 = miller[3 * p + 1], n2 = miller[3 * p + 2];
        /* (h^-T n)_a = sum_b hinv[b][a] n_b */
        for (int a = 0; a < 3; ++a)
            q_out[3 * p + a] = two_pi * (hi[0 * 3 + a] * n0 + hi[1 * 3 + a] * n1 + hi[2 * 3 + a] * n2);
    }
    return 1;
}

/*
 * Complex amplitude S(q,t) = sum_j f_j exp(+i q.r_j(t)) for every frame and
 * every listed Miller index.
 *   pos     float32 [n_frames][n_atoms][3]
 *   f       float64 [n_atoms]
 *   h       float64 [9]   row-major cell matrix (columns = edge vectors)
 *   miller  int32 [n_q][3]
 *   amp_out float64 [n_frames][n_q][2]   (re, im)
 * Returns 1 on success, 0 for a singular cell.
 */
int oracle_amplitude(const float* pos, int64_t n_atoms, int64_t n_frames, const double* f,
                     const double* h, const int32_t* miller, int64_t n_q, double* amp_out,
                     int n_threads) {
    double* q = (double*)0;
    /* small fixed-size path keeps this file free of allocation helpers */
    enum { QCHUNK = 1024 };
    double qbuf[QCHUNK * 3];
    /* n_threads > 0 applies to this call only (no global OpenMP setting) */
#ifdef _OPENMP
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
#endif
    for (int64_t q0 = 0; q0 < n_q; q0 += QCHUNK) {
        int64_t nq = n_q - q0 < QCHUNK ? n_q - q0 : QCHUNK;
        if (!oracle_qvectors(h, miller + 3 * q0, nq, qbuf)) return 0;
        q = qbuf;
        int64_t total = n_frames * nq;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
        for (int64_t w = 0; w < total; ++w) {
            int64_t t = w / nq, p = w % nq;
            const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
            const float* r = pos + (size_t)t * (size_t)n_atoms * 3;
            neumaier re = {0.0, 0.0}, im = {0.0, 0.0};
            for (int64_t j = 0; j < n_atoms; ++j) {
                double th = qx * (double)r[3 * j] + qy * (double)r[3 * j + 1] + qz * (double)r[3 * j + 2];
                nm_add(&re, f[j] * cos(th));
                nm_add(&im, f[j] * sin(th));
            }
            double* o = amp_out + ((size_t)t * (size_t)n_q + (size_t)(q0 + p)) * 2;
            o[0] = nm_value(&re);
            o[1] = nm_value(&im);
        }
    }
    return 1;
}

/* I(q,t) = |S(q,t)|^2 from the amplitude above; I_out float64 [n_frames][n_q] */
int oracle_intensity(const float* pos, int64_t n_atoms, int64_t n_frames, const double* f,
                     const double* h, const int32_t* miller, int64_t n_q, double* amp_scratch,
                     double* I_out, int n_threads) {
    if (!oracle_amplitude(pos, n_atoms, n_frames, f, h, miller, n_q, amp_scratch, n_threads)) return 0;
    for (int64_t k = 0; k < n_frames * n_q; ++k) {
        double a = amp_scratch[2 * k], b = amp_scratch[2 * k + 1];
        I_out[k] = a * a + b * b;
    }
    return 1;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
