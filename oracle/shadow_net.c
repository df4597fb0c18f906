/*
 * FP64 CPU oracle of the learned shadow-transmittance surrogate.
 *
 * TEST INFRASTRUCTURE ONLY, like mrf_oracle.c: the plain definition the CUDA
 * training and inference kernels are checked against.  The renderer never
 * calls it and shares no code with it.
 *
 * The paper's shadow rays (Sec. 3.1, "Shadow rays") take the field's
 * transmittance exp(-int sigma) from a shading point toward a light.  The
 * surrogate replaces that march by a small network of the point and the
 * direction toward the light:
 *   input   : the point in the field's local frame, scaled to [0,1]^3 by the
 *             field box, encoded by a multiresolution hash grid (the encoding
 *             the paper's field uses, here with n_levels levels of 2 FP32
 *             features, resolutions level_res[l], table 2^log2_T entries per
 *             level: dense index when (N+1)^3 fits, else the spatial hash with
 *             primes 1, 2654435761, 805459861), concatenated with the real
 *             spherical harmonics of bands 0..3 of the direction (16 values);
 *   network : 32 -> 64 ReLU -> 64 ReLU -> 64 ReLU -> 1, T = sigmoid(z);
 *   loss    : mean squared error against the marched transmittance.
 * Parameters, one flat vector: the table (level-major, entry-major, 2
 * features), then W1 (64 x 32, row-major), b1, W2 (64 x 64), b2, W3, b3,
 * W4 (64), b4 (1).
 *
 * The gradient is back-propagation written out layer by layer; the tests pin
 * it to central finite differences of the loss.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <string.h>

#define SN_W 64
#define SN_IN 32

typedef struct orc_snet {
    uint32_t n_levels, log2_T;
    const uint32_t *level_res;
    float aabb_min[3], aabb_max[3];
    const float *field_pose;   /* 3x4 local-to-world [R | t], NULL = identity */
    const double *params;
} orc_snet;

static uint64_t sn_table_size(const orc_snet *n) { return (uint64_t)n->n_levels << n->log2_T; }

uint64_t orc_snet_n_params(const orc_snet *n) {
    return sn_table_size(n) * 2 + (uint64_t)SN_W * SN_IN + SN_W + 2ull * (SN_W * SN_W + SN_W) + SN_W + 1;
}

/* Real spherical harmonics of bands l = 0..3 at the unit direction w,
 * orthonormal on the sphere, in the order (l, m = -l..l). */
void orc_sh16(const double w[3], double Y[16]) {
    const double x = w[0], y = w[1], z = w[2], pi = M_PI;
    Y[0] = 0.5 * sqrt(1.0 / pi);
    const double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
    const double c2 = 0.5 * sqrt(15.0 / pi);
    Y[4] = c2 * x * y;
    Y[5] = c2 * y * z;
    Y[6] = 0.25 * sqrt(5.0 / pi) * (3.0 * z * z - 1.0);
    Y[7] = c2 * x * z;
    Y[8] = 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
    Y[9] = 0.25 * sqrt(35.0 / (2.0 * pi)) * y * (3.0 * x * x - y * y);
    Y[10] = 0.5 * sqrt(105.0 / pi) * x * y * z;
    Y[11] = 0.25 * sqrt(21.0 / (2.0 * pi)) * y * (5.0 * z * z - 1.0);
    Y[12] = 0.25 * sqrt(7.0 / pi) * (5.0 * z * z * z - 3.0 * z);
    Y[13] = 0.25 * sqrt(21.0 / (2.0 * pi)) * x * (5.0 * z * z - 1.0);
    Y[14] = 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
    Y[15] = 0.25 * sqrt(35.0 / (2.0 * pi)) * x * (x * x - 3.0 * y * y);
}

/* world point / direction to the field's local frame (inverse of the pose) */
static void sn_local(const orc_snet *n, const double p[3], const double w[3], double pl[3], double wl[3]) {
    if (!n->field_pose) {
        memcpy(pl, p, 3 * sizeof(double));
        memcpy(wl, w, 3 * sizeof(double));
        return;
    }
    const float *M = n->field_pose;
    double q[3];
    for (int a = 0; a < 3; ++a) q[a] = p[a] - M[4 * a + 3];
    for (int a = 0; a < 3; ++a) {
        pl[a] = M[a] * q[0] + M[4 + a] * q[1] + M[8 + a] * q[2];        /* R^T (p - t) */
        wl[a] = M[a] * w[0] + M[4 + a] * w[1] + M[8 + a] * w[2];
    }
}

/* Corner indices and trilinear weights of level l at the local point pl. */
static void sn_corners(const orc_snet *n, uint32_t l, const double pl[3], uint64_t idx[8], double wt[8]) {
    const uint64_t T = 1ull << n->log2_T;
    const uint32_t N = n->level_res[l];
    const int dense = (uint64_t)(N + 1) * (N + 1) * (N + 1) <= T;
    int64_t c[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = (pl[a] - n->aabb_min[a]) / ((double)n->aabb_max[a] - n->aabb_min[a]);
        if (u < 0.0) u = 0.0;
        if (u > 1.0) u = 1.0;
        u *= N;
        double fl = floor(u);
        if (fl > N - 1) fl = N - 1;
        c[a] = (int64_t)fl;
        f[a] = u - fl;
    }
    for (int k = 0; k < 8; ++k) {
        uint32_t x = (uint32_t)(c[0] + (k & 1)), y = (uint32_t)(c[1] + ((k >> 1) & 1)),
                 z = (uint32_t)(c[2] + ((k >> 2) & 1));
        wt[k] = ((k & 1) ? f[0] : 1.0 - f[0]) * (((k >> 1) & 1) ? f[1] : 1.0 - f[1]) *
                (((k >> 2) & 1) ? f[2] : 1.0 - f[2]);
        uint64_t i;
        if (dense) i = x + (uint64_t)(N + 1) * (y + (uint64_t)(N + 1) * z);
        else i = (uint32_t)(x * 1u ^ y * 2654435761u ^ z * 805459861u) & (uint32_t)(T - 1);
        idx[k] = (uint64_t)l * T + i;
    }
}

/* The 32 inputs: hash features (level-major, 2 per level; the first 16) and
 * the 16 spherical harmonics.  Requires n_levels == 8. */
void orc_snet_encode(const orc_snet *n, const double p[3], const double w[3], double x[SN_IN]) {
    double pl[3], wl[3];
    sn_local(n, p, w, pl, wl);
    for (uint32_t l = 0; l < n->n_levels; ++l) {
        uint64_t idx[8];
        double wt[8];
        sn_corners(n, l, pl, idx, wt);
        x[2 * l] = x[2 * l + 1] = 0.0;
        for (int k = 0; k < 8; ++k) {
            x[2 * l] += wt[k] * n->params[2 * idx[k]];
            x[2 * l + 1] += wt[k] * n->params[2 * idx[k] + 1];
        }
    }
    double wn = sqrt(wl[0] * wl[0] + wl[1] * wl[1] + wl[2] * wl[2]);
    double u[3] = {wl[0] / wn, wl[1] / wn, wl[2] / wn};
    orc_sh16(u, x + 2 * n->n_levels);
}

typedef struct {
    double x[SN_IN], a1[SN_W], h1[SN_W], a2[SN_W], h2[SN_W], a3[SN_W], h3[SN_W], z, T;
} sn_act;

static void sn_forward(const orc_snet *n, const double p[3], const double w[3], sn_act *A) {
    const double *P = n->params + 2 * sn_table_size(n);
    const double *W1 = P, *b1 = W1 + SN_W * SN_IN, *W2 = b1 + SN_W, *b2 = W2 + SN_W * SN_W, *W3 = b2 + SN_W,
                 *b3 = W3 + SN_W * SN_W, *W4 = b3 + SN_W, *b4 = W4 + SN_W;
    orc_snet_encode(n, p, w, A->x);
    for (int i = 0; i < SN_W; ++i) {
        double s = b1[i];
        for (int k = 0; k < SN_IN; ++k) s += W1[i * SN_IN + k] * A->x[k];
        A->a1[i] = s;
        A->h1[i] = s > 0 ? s : 0;
    }
    for (int i = 0; i < SN_W; ++i) {
        double s = b2[i];
        for (int k = 0; k < SN_W; ++k) s += W2[i * SN_W + k] * A->h1[k];
        A->a2[i] = s;
        A->h2[i] = s > 0 ? s : 0;
    }
    for (int i = 0; i < SN_W; ++i) {
        double s = b3[i];
        for (int k = 0; k < SN_W; ++k) s += W3[i * SN_W + k] * A->h2[k];
        A->a3[i] = s;
        A->h3[i] = s > 0 ? s : 0;
    }
    double z = b4[0];
    for (int k = 0; k < SN_W; ++k) z += W4[k] * A->h3[k];
    A->z = z;
    A->T = 1.0 / (1.0 + exp(-z));
}

/* Smallest |pre-activation| over the hidden units at (p, w): where it is at
 * rounding level, FP32 and FP64 may take different ReLU branches and their
 * gradients legitimately differ (the network's ambiguity margin). */
double orc_snet_relu_margin(const orc_snet *n, const double p[3], const double w[3]) {
    sn_act A;
    sn_forward(n, p, w, &A);
    double m = INFINITY;
    for (int i = 0; i < SN_W; ++i) {
        if (fabs(A.a1[i]) < m) m = fabs(A.a1[i]);
        if (fabs(A.a2[i]) < m) m = fabs(A.a2[i]);
        if (fabs(A.a3[i]) < m) m = fabs(A.a3[i]);
    }
    return m;
}

/* Surrogate transmittance from world point p along world direction w. */
double orc_snet_forward(const orc_snet *n, const double p[3], const double w[3]) {
    sn_act A;
    sn_forward(n, p, w, &A);
    return A.T;
}

/* Loss (1/m) sum_i (T(p_i, w_i) - y_i)^2 over the m pairs (pw: m x 6 = point,
 * direction) and, if grad is non-NULL, its gradient with respect to every
 * parameter (grad: orc_snet_n_params values, overwritten). */
double orc_snet_loss_grad(const orc_snet *n, const double *pw, const double *y, uint32_t m, double *grad) {
    const uint64_t tbl = 2 * sn_table_size(n);
    const double *P = n->params + tbl;
    const double *W1 = P, *W2 = W1 + SN_W * SN_IN + SN_W, *W3 = W2 + SN_W * SN_W + SN_W,
                 *W4 = W3 + SN_W * SN_W + SN_W;
    if (grad) memset(grad, 0, orc_snet_n_params(n) * sizeof(double));
    double *g = grad ? grad + tbl : NULL;
    double *gW1 = g, *gb1 = g ? gW1 + SN_W * SN_IN : NULL, *gW2 = g ? gb1 + SN_W : NULL,
           *gb2 = g ? gW2 + SN_W * SN_W : NULL, *gW3 = g ? gb2 + SN_W : NULL, *gb3 = g ? gW3 + SN_W * SN_W : NULL,
           *gW4 = g ? gb3 + SN_W : NULL, *gb4 = g ? gW4 + SN_W : NULL;
    double loss = 0.0;
    for (uint32_t s = 0; s < m; ++s) {
        sn_act A;
        sn_forward(n, pw + 6 * s, pw + 6 * s + 3, &A);
        const double r = A.T - y[s];
        loss += r * r / m;
        if (!grad) continue;
        /* dL/dz = 2 r / m * T (1 - T) */
        const double dz = 2.0 * r / m * A.T * (1.0 - A.T);
        double d3[SN_W], d2[SN_W], d1[SN_W], dx[SN_IN];
        gb4[0] += dz;
        for (int k = 0; k < SN_W; ++k) {
            gW4[k] += dz * A.h3[k];
            d3[k] = A.a3[k] > 0 ? dz * W4[k] : 0.0;
        }
        for (int k = 0; k < SN_W; ++k) {
            double s2 = 0.0;
            for (int i = 0; i < SN_W; ++i) s2 += W3[i * SN_W + k] * d3[i];
            d2[k] = A.a2[k] > 0 ? s2 : 0.0;
        }
        for (int i = 0; i < SN_W; ++i) {
            gb3[i] += d3[i];
            for (int k = 0; k < SN_W; ++k) gW3[i * SN_W + k] += d3[i] * A.h2[k];
        }
        for (int k = 0; k < SN_W; ++k) {
            double s1 = 0.0;
            for (int i = 0; i < SN_W; ++i) s1 += W2[i * SN_W + k] * d2[i];
            d1[k] = A.a1[k] > 0 ? s1 : 0.0;
        }
        for (int i = 0; i < SN_W; ++i) {
            gb2[i] += d2[i];
            for (int k = 0; k < SN_W; ++k) gW2[i * SN_W + k] += d2[i] * A.h1[k];
        }
        for (int k = 0; k < SN_IN; ++k) {
            double s0 = 0.0;
            for (int i = 0; i < SN_W; ++i) s0 += W1[i * SN_IN + k] * d1[i];
            dx[k] = s0;
        }
        for (int i = 0; i < SN_W; ++i) {
            gb1[i] += d1[i];
            for (int k = 0; k < SN_IN; ++k) gW1[i * SN_IN + k] += d1[i] * A.x[k];
        }
        /* the hash features are trilinear in the table entries */
        double pl[3], wl[3];
        sn_local(n, pw + 6 * s, pw + 6 * s + 3, pl, wl);
        for (uint32_t l = 0; l < n->n_levels; ++l) {
            uint64_t idx[8];
            double wt[8];
            sn_corners(n, l, pl, idx, wt);
            for (int k = 0; k < 8; ++k) {
                grad[2 * idx[k]] += wt[k] * dx[2 * l];
                grad[2 * idx[k] + 1] += wt[k] * dx[2 * l + 1];
            }
        }
    }
    return loss;
}

/* One Adam step (Kingma and Ba, ICLR 2015, Algorithm 1) at step number t >= 1:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * theta -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void orc_adam_step(double *theta, double *m, double *v, const double *g, uint64_t n, uint32_t t, double lr, double b1,
                   double b2, double eps) {
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (uint64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
