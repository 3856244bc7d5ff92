/*
 * net_oracle.c -- plain FP64 CPU oracle for the learned post-smoother that may replace the
 * dropped post-smoothing of the (1,0) SMG cycle inside flexible PCG (not part of arXiv:1212.6680;
 * flexible PCG, eq. (2), is what tolerates such a nonlinear preconditioner).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite and nothing in the product library.
 *
 * Reading (the paper is silent on all of it):
 *   network   conv 1 -> 16 -> 16 -> 1 channels, 3x3x3 kernels, zero padding (the homogeneous
 *             Dirichlet boundary), no bias, ReLU after the first two layers; positively
 *             homogeneous: Net(c x) = c Net(x) for c > 0.
 *   scaling   delta = rms(rho) * Net(rho / rms(rho)), rms = sqrt(sum rho^2 / N); delta = 0 when
 *             rho = 0.  The correction is then scale-equivariant in the residual.
 *   weights   one array of 7776 doubles: layer 1 [16][1][27], layer 2 [16][16][27],
 *             layer 3 [1][16][27], each [out channel][in channel][tap]; tap
 *             t = (dz+1)*9 + (dy+1)*3 + (dx+1) weights the input at (x+dx, y+dy, z+dz).
 *   loss      energy norm of the remaining error relative to the target:
 *             L = (e - delta)^T A (e - delta) / e^T A e.
 *   use       s0 = T r (the (1,0) cycle), rho = r - A s0, delta = Net-correction(rho);
 *             s = s0 + delta when ||rho - A delta||_2 < ||rho||_2, else s = s0 (the judge).
 *
 * Activations are channel-major: a[c][(z*ny + y)*nx + x].
 *
 * Optionally (act_bf16 = 1) the two hidden activations are rounded to BF16 after the ReLU, as a
 * BF16 implementation stores them; the ReLU masks of the backward pass then follow the rounded
 * values.  Everything else stays FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "smg_oracle.h"

static size_t npts(int nx, int ny, int nz) { return (size_t)nx * (size_t)ny * (size_t)nz; }

/* out[co][p] = sum_ci sum_t w[co][ci][t] * in[ci][p + off_t]  (zero outside the brick) */
void orc_conv3d(int nx, int ny, int nz, int cin, int cout, const double *w, const double *in, double *out)
{
    size_t n = npts(nx, ny, nz);
    for (int co = 0; co < cout; ++co)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double acc = 0.0;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dz = -1; dz <= 1; ++dz)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    int xx = x + dx, yy = y + dy, zz = z + dz;
                                    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                                    int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                                    acc += w[((size_t)co * cin + ci) * 27 + t] *
                                           in[(size_t)ci * n + ((size_t)zz * ny + yy) * nx + xx];
                                }
                    out[(size_t)co * n + ((size_t)z * ny + y) * nx + x] = acc;
                }
}

/* The adjoint of orc_conv3d in its input: gin[ci][q] = sum_co sum_t w[co][ci][t] gout[co][q - off_t]. */
void orc_conv3d_adj(int nx, int ny, int nz, int cin, int cout, const double *w, const double *gout, double *gin)
{
    size_t n = npts(nx, ny, nz);
    memset(gin, 0, sizeof(double) * n * (size_t)cin);
    for (int co = 0; co < cout; ++co)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    double g = gout[(size_t)co * n + ((size_t)z * ny + y) * nx + x];
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dz = -1; dz <= 1; ++dz)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    int xx = x + dx, yy = y + dy, zz = z + dz;
                                    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                                    int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                                    gin[(size_t)ci * n + ((size_t)zz * ny + yy) * nx + xx] +=
                                        w[((size_t)co * cin + ci) * 27 + t] * g;
                                }
                }
}

/* Gradient of sum_co <gout[co], out[co]> in the weights: gw[co][ci][t] = sum_p gout[co][p] in[ci][p + off_t]. */
void orc_conv3d_wgrad(int nx, int ny, int nz, int cin, int cout, const double *in, const double *gout, double *gw)
{
    size_t n = npts(nx, ny, nz);
    for (int co = 0; co < cout; ++co)
        for (int ci = 0; ci < cin; ++ci)
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        double acc = 0.0;
                        for (int z = 0; z < nz; ++z)
                            for (int y = 0; y < ny; ++y)
                                for (int x = 0; x < nx; ++x) {
                                    int xx = x + dx, yy = y + dy, zz = z + dz;
                                    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) continue;
                                    acc += gout[(size_t)co * n + ((size_t)z * ny + y) * nx + x] *
                                           in[(size_t)ci * n + ((size_t)zz * ny + yy) * nx + xx];
                                }
                        int t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                        gw[((size_t)co * cin + ci) * 27 + t] = acc;
                    }
}

/* IEEE binary32 rounding of v, then rounding to the nearest BF16 (8 significant bits), ties to
 * even: the upper 16 bits of the binary32 after adding half an ulp of BF16 (0x7FFF plus the
 * lowest kept bit). */
double orc_round_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof(u));
    u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, sizeof(f));
    return (double)f;
}

#define NET_C 16
#define NET_W1 0
#define NET_W2 (NET_C * 27)
#define NET_W3 (NET_W2 + NET_C * NET_C * 27)

static double rms_of(size_t n, const double *v)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += v[i] * v[i];
    return sqrt(s / (double)n);
}

/* Forward pass keeping the pre-activations (h1, h2: NET_C*N each) for the backward pass. */
static double net_forward_keep(int nx, int ny, int nz, const double *w, const double *rho, double *x0, double *h1,
                               double *a1, double *h2, double *a2, double *y, int act_bf16)
{
    size_t n = npts(nx, ny, nz);
    double rms = rms_of(n, rho);
    double inv = rms > 0.0 ? 1.0 / rms : 0.0;
    for (size_t i = 0; i < n; ++i) x0[i] = rho[i] * inv;
    orc_conv3d(nx, ny, nz, 1, NET_C, w + NET_W1, x0, h1);
    for (size_t i = 0; i < n * NET_C; ++i) {
        a1[i] = h1[i] > 0.0 ? h1[i] : 0.0;
        if (act_bf16) a1[i] = orc_round_bf16(a1[i]);
    }
    orc_conv3d(nx, ny, nz, NET_C, NET_C, w + NET_W2, a1, h2);
    for (size_t i = 0; i < n * NET_C; ++i) {
        a2[i] = h2[i] > 0.0 ? h2[i] : 0.0;
        if (act_bf16) a2[i] = orc_round_bf16(a2[i]);
    }
    orc_conv3d(nx, ny, nz, NET_C, 1, w + NET_W3, a2, y);
    return rms;
}

void orc_net_forward(int nx, int ny, int nz, const double *w, const double *rho, double *delta)
{
    orc_net_forward_ex(nx, ny, nz, w, rho, delta, 0);
}

void orc_net_forward_ex(int nx, int ny, int nz, const double *w, const double *rho, double *delta, int act_bf16)
{
    size_t n = npts(nx, ny, nz);
    double *x0 = (double *)malloc(sizeof(double) * n);
    double *h1 = (double *)malloc(sizeof(double) * n * NET_C);
    double *a1 = (double *)malloc(sizeof(double) * n * NET_C);
    double *h2 = (double *)malloc(sizeof(double) * n * NET_C);
    double *a2 = (double *)malloc(sizeof(double) * n * NET_C);
    double rms = net_forward_keep(nx, ny, nz, w, rho, x0, h1, a1, h2, a2, delta, act_bf16);
    for (size_t i = 0; i < n; ++i) delta[i] *= rms;
    free(x0);
    free(h1);
    free(a1);
    free(h2);
    free(a2);
}

double orc_net_loss_grad(int nx, int ny, int nz, const double *w, const double *rho, const double *e, double *grad)
{
    return orc_net_loss_grad_ex(nx, ny, nz, w, rho, e, grad, 0);
}

double orc_net_loss_grad_ex(int nx, int ny, int nz, const double *w, const double *rho, const double *e, double *grad,
                            int act_bf16)
{
    size_t n = npts(nx, ny, nz);
    double *x0 = (double *)malloc(sizeof(double) * n);
    double *h1 = (double *)malloc(sizeof(double) * n * NET_C);
    double *a1 = (double *)malloc(sizeof(double) * n * NET_C);
    double *h2 = (double *)malloc(sizeof(double) * n * NET_C);
    double *a2 = (double *)malloc(sizeof(double) * n * NET_C);
    double *y = (double *)malloc(sizeof(double) * n);
    double *d = (double *)malloc(sizeof(double) * n);
    double *Ad = (double *)malloc(sizeof(double) * n);
    double *Ae = (double *)malloc(sizeof(double) * n);
    double *gy = (double *)malloc(sizeof(double) * n);
    double *ga = (double *)malloc(sizeof(double) * n * NET_C);
    double *gh = (double *)malloc(sizeof(double) * n * NET_C);

    double rms = net_forward_keep(nx, ny, nz, w, rho, x0, h1, a1, h2, a2, y, act_bf16);
    for (size_t i = 0; i < n; ++i) d[i] = e[i] - rms * y[i];
    orc_apply_A(nx, ny, nz, d, Ad);
    orc_apply_A(nx, ny, nz, e, Ae);
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < n; ++i) {
        num += d[i] * Ad[i];
        den += e[i] * Ae[i];
    }
    double loss = den > 0.0 ? num / den : 0.0;
    if (grad) {
        /* dL/d delta = -2 A d / e^T A e (A symmetric); delta = rms * y */
        double sc = den > 0.0 ? -2.0 * rms / den : 0.0;
        for (size_t i = 0; i < n; ++i) gy[i] = sc * Ad[i];
        orc_conv3d_wgrad(nx, ny, nz, NET_C, 1, a2, gy, grad + NET_W3);
        orc_conv3d_adj(nx, ny, nz, NET_C, 1, w + NET_W3, gy, ga);
        for (size_t i = 0; i < n * NET_C; ++i) gh[i] = a2[i] > 0.0 ? ga[i] : 0.0;
        orc_conv3d_wgrad(nx, ny, nz, NET_C, NET_C, a1, gh, grad + NET_W2);
        orc_conv3d_adj(nx, ny, nz, NET_C, NET_C, w + NET_W2, gh, ga);
        for (size_t i = 0; i < n * NET_C; ++i) gh[i] = a1[i] > 0.0 ? ga[i] : 0.0;
        orc_conv3d_wgrad(nx, ny, nz, 1, NET_C, x0, gh, grad + NET_W1);
    }
    free(x0);
    free(h1);
    free(a1);
    free(h2);
    free(a2);
    free(y);
    free(d);
    free(Ad);
    free(Ae);
    free(gy);
    free(ga);
    free(gh);
    return loss;
}

int orc_learned_correct(int nx, int ny, int nz, const double *w, const double *r, double *s)
{
    size_t n = npts(nx, ny, nz);
    double *rho = (double *)malloc(sizeof(double) * n);
    double *delta = (double *)malloc(sizeof(double) * n);
    double *t = (double *)malloc(sizeof(double) * n);
    orc_apply_A(nx, ny, nz, s, t);
    for (size_t i = 0; i < n; ++i) rho[i] = r[i] - t[i];
    orc_net_forward(nx, ny, nz, w, rho, delta);
    orc_apply_A(nx, ny, nz, delta, t);
    double before = 0.0, after = 0.0;
    for (size_t i = 0; i < n; ++i) {
        before += rho[i] * rho[i];
        after += (rho[i] - t[i]) * (rho[i] - t[i]);
    }
    int accepted = after < before;
    if (accepted)
        for (size_t i = 0; i < n; ++i) s[i] += delta[i];
    free(rho);
    free(delta);
    free(t);
    return accepted;
}
