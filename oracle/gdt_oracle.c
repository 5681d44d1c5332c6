/*
 * Oracle for the generalised geodesic distance transform computed by
 * parallelisable raster-scan passes (FastGeodis, Implementation section;
 * Criminisi et al. 2009 scan, Criminisi et al. 2008 generalised GDT).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, sequential CPU
 * restatement of the method used to check the CUDA path.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header or table with the CUDA library.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fopenmp -fPIC -shared
 * (no -march flags: no FMA contraction, no flush-to-zero).
 *
 * Layout: image [B][C][D][H][W], mask and dist [B][D][H][W], contiguous;
 * 2D inputs use D = 1.  codes [iterations * passes][B][D*H*W] bytes.
 *
 * Pins: see the oracle tests (Dijkstra on the 8/26-connected grid at the
 * fixed point, closed-form chamfer and total-variation cases, invariants,
 * brute force on 1D and tiny inputs, finite differences for the backward).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REAL float
#define SUFFIX f32
#define SQRT sqrtf
#define FMIN fminf
#include "gdt_core.inc"
#undef REAL
#undef SUFFIX
#undef SQRT
#undef FMIN

#define REAL double
#define SUFFIX f64
#define SQRT sqrt
#define FMIN fmin
#include "gdt_core.inc"
#undef REAL
#undef SUFFIX
#undef SQRT
#undef FMIN

/* The paper's pass order (Implementation section).  Axis 0 = D, 1 = H, 2 = W;
 * direction +1 sweeps towards larger indices. */
static const int SCHED_2D[8] = {1, +1, 1, -1, 2, +1, 2, -1};           /* TB BT LR RL */
static const int SCHED_3D[12] = {0, +1, 0, -1, 1, +1, 1, -1, 2, +1, 2, -1}; /* FB BF TB BT LR RL */

static int check_common(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W) {
    if (ndim != 2 && ndim != 3) return -1;
    if (B < 0 || C < 1 || D < 0 || H < 0 || W < 0) return -1;
    if (ndim == 2 && D != 1) return -1;
    return 0;
}

int oracle_num_passes(int ndim) { return ndim == 3 ? 6 : 4; }

/* Forward transform, paper schedule, in float.  spacing = (sD, sH, sW); 2D
 * callers pass (1, 1, 1).  nthreads > 1 parallelises over the elements of a
 * line (the CPU design the paper describes); results do not depend on it. */
int oracle_gdt_f32(const float* image, const float* mask, float* dist, int ndim, int64_t B,
                   int64_t C, int64_t D, int64_t H, int64_t W, const float* spacing, float v,
                   float lambda, int iterations, uint8_t* codes, int nthreads) {
    if (check_common(ndim, B, C, D, H, W) || iterations < 0) return -1;
    const int64_t ext[3] = {D, H, W};
    const int64_t N = D * H * W;
    for (int64_t i = 0; i < B * N; ++i) dist[i] = v * mask[i];
    return run_schedule_f32(ndim, image, dist, B, C, ext, spacing, lambda,
                            ndim == 3 ? SCHED_3D : SCHED_2D, oracle_num_passes(ndim),
                            iterations, codes, nthreads, NULL);
}

int oracle_gdt_f64(const double* image, const double* mask, double* dist, int ndim, int64_t B,
                   int64_t C, int64_t D, int64_t H, int64_t W, const double* spacing, double v,
                   double lambda, int iterations, uint8_t* codes) {
    if (check_common(ndim, B, C, D, H, W) || iterations < 0) return -1;
    const int64_t ext[3] = {D, H, W};
    const int64_t N = D * H * W;
    for (int64_t i = 0; i < B * N; ++i) dist[i] = v * mask[i];
    return run_schedule_f64(ndim, image, dist, B, C, ext, spacing, lambda,
                            ndim == 3 ? SCHED_3D : SCHED_2D, oracle_num_passes(ndim),
                            iterations, codes, 1, NULL);
}

/* Forward with an arbitrary schedule of (axis, direction) pairs, in double.
 * iterations < 0 repeats until a whole iteration leaves dist unchanged (the
 * fixed point); the count is returned in *iters_run. */
int oracle_gdt_sched_f64(const double* image, const double* mask, double* dist, int ndim,
                         int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                         const double* spacing, double v, double lambda, const int* sched,
                         int npass, int iterations, int* iters_run) {
    if (check_common(ndim, B, C, D, H, W)) return -1;
    for (int i = 0; i < npass; ++i) {
        if (sched[2 * i] < 0 || sched[2 * i] > 2 || (sched[2 * i + 1] != 1 && sched[2 * i + 1] != -1))
            return -1;
        if (ndim == 2 && sched[2 * i] == 0) return -1;
    }
    const int64_t ext[3] = {D, H, W};
    const int64_t N = D * H * W;
    for (int64_t i = 0; i < B * N; ++i) dist[i] = v * mask[i];
    return run_schedule_f64(ndim, image, dist, B, C, ext, spacing, lambda, sched, npass,
                            iterations, NULL, 1, iters_run);
}

/* Backward through recorded codes (see gdt_core.inc).  grad_dist is read
 * only; grad_image, grad_mask, lambda_terms and v_terms (all nullable; v_terms
 * needs mask) are written. */
int oracle_backward_f32(const float* grad_dist, const float* image, const uint8_t* codes,
                        float* grad_image, float* grad_mask, int ndim, int64_t B, int64_t C,
                        int64_t D, int64_t H, int64_t W, const float* spacing, float v,
                        float lambda, int iterations, const float* mask, float* lambda_terms,
                        float* v_terms) {
    if (v_terms && !mask) return -1;
    if (check_common(ndim, B, C, D, H, W) || iterations < 0) return -1;
    const int64_t ext[3] = {D, H, W};
    const int64_t N = D * H * W;
    float* G = (float*)malloc((size_t)(B * N) * sizeof(float));
    if (!G) return -2;
    memcpy(G, grad_dist, (size_t)(B * N) * sizeof(float));
    int r = backward_f32(ndim, image, codes, G, grad_image, grad_mask, B, C, ext, spacing, v,
                         lambda, ndim == 3 ? SCHED_3D : SCHED_2D, oracle_num_passes(ndim),
                         iterations, mask, lambda_terms, v_terms);
    free(G);
    return r;
}

int oracle_backward_f64(const double* grad_dist, const double* image, const uint8_t* codes,
                        double* grad_image, double* grad_mask, int ndim, int64_t B, int64_t C,
                        int64_t D, int64_t H, int64_t W, const double* spacing, double v,
                        double lambda, int iterations, const double* mask, double* lambda_terms,
                        double* v_terms) {
    if (v_terms && !mask) return -1;
    if (check_common(ndim, B, C, D, H, W) || iterations < 0) return -1;
    const int64_t ext[3] = {D, H, W};
    const int64_t N = D * H * W;
    double* G = (double*)malloc((size_t)(B * N) * sizeof(double));
    if (!G) return -2;
    memcpy(G, grad_dist, (size_t)(B * N) * sizeof(double));
    int r = backward_f64(ndim, image, codes, G, grad_image, grad_mask, B, C, ext, spacing, v,
                         lambda, ndim == 3 ? SCHED_3D : SCHED_2D, oracle_num_passes(ndim),
                         iterations, mask, lambda_terms, v_terms);
    free(G);
    return r;
}
