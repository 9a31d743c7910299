/*
 * Oracle: the path-guiding proposal in FP64. The paper has no learned
 * component (its nearest relatives are the static light hierarchy of
 * Sec. 2.1.1, the environment pyramid of Sec. 2.1.2 and photon aiming of
 * Sec. 2.1.3); this file follows textbook definitions only:
 *   - von Mises-Fisher lobe on the sphere, q(w) = k/(2 pi (1 - e^{-2k}))
 *     exp(k (mu.w - 1)), sampled as in Jakob 2012 ("Numerically stable
 *     sampling of the von Mises Fisher distribution on S2");
 *   - one-blob input encoding (Mueller et al. 2019): 32 Gaussian bins per
 *     scalar in [0,1], sigma = 1/32, evaluated at the bin centres;
 *   - multilayer perceptron 224 -> 64 -> 64 -> 64 -> 64 -> 40, ReLU on the
 *     four hidden layers, no biases, weights stored [out][in] row-major, layer
 *     after layer;
 *   - 40 outputs = 8 lobes x (mu 3: normalised, kappa 1: softplus clamped to
 *     [1e-2, 1e4], logit 1: softmax over lobes);
 *   - loss = mean over the batch of -weight * log q_mix(wi), weight = F/p
 *     (the sampled contribution over the proposal density);
 *   - Adam (Kingma and Ba 2015) with bias correction.
 * The paper has no passage for any of this, so no printed value can pin it;
 * every function is pinned instead to what the mathematics fixes
 * (tests/test_oracle_guide.py): the vMF density integrates to one and its
 * samples have the closed-form mean cosine, the mixture integrates to one,
 * the one-blob bins equal their closed form, the forward pass equals plain
 * matrix products, the gradients equal central differences of the loss, and
 * the first Adam steps equal the textbook update.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define KMIN 1e-2
#define KMAX 1e4

static const int g_dims[6] = {OR_GUIDE_IN, OR_GUIDE_HID, OR_GUIDE_HID, OR_GUIDE_HID, OR_GUIDE_HID, OR_GUIDE_OUT};

int64_t or_guide_nparams(void) {
    int64_t n = 0;
    for (int l = 0; l < 5; ++l) n += (int64_t)g_dims[l] * g_dims[l + 1];
    return n;
}

double or_vmf_pdf(double kappa, const double mu[3], const double w[3]) {
    double c = mu[0] * w[0] + mu[1] * w[1] + mu[2] * w[2];
    return kappa / (2.0 * OR_PI * (1.0 - exp(-2.0 * kappa))) * exp(kappa * (c - 1.0));
}

void or_vmf_sample(double kappa, const double mu[3], double u1, double u2,
                   double w[3]) {
    double ct = 1.0 + log(u1 + (1.0 - u1) * exp(-2.0 * kappa)) / kappa;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double phi = 2.0 * OR_PI * u2;
    double t[3], b[3];
    or_onb(mu, t, b);
    for (int a = 0; a < 3; ++a)
        w[a] = st * cos(phi) * t[a] + st * sin(phi) * b[a] + ct * mu[a];
}

void or_oneblob(const double s[7], double *enc) {
    const double sig = 1.0 / OR_GUIDE_BINS;
    for (int i = 0; i < 7; ++i)
        for (int c = 0; c < OR_GUIDE_BINS; ++c) {
            double dlt = s[i] - ((double)c + 0.5) / OR_GUIDE_BINS;
            enc[i * OR_GUIDE_BINS + c] = exp(-dlt * dlt / (2.0 * sig * sig));
        }
}

static void dir_features(const double w[3], double *a, double *b) {
    double cy = fmax(-1.0, fmin(1.0, w[1]));
    double phi = atan2(w[2], w[0]);
    if (phi < 0.0) phi += 2.0 * OR_PI;
    *a = 0.5 * (cy + 1.0);
    *b = phi / (2.0 * OR_PI);
}

void or_guide_features(const double pos01[3], const double wo[3],
                       const double n[3], double s[7]) {
    for (int a = 0; a < 3; ++a) s[a] = fmin(1.0, fmax(0.0, pos01[a]));
    dir_features(wo, &s[3], &s[4]);
    dir_features(n, &s[5], &s[6]);
}

/* acts (if not NULL) receives, per sample, the post-ReLU activations of the
 * four hidden layers (4 x 64). */
void or_mlp_forward(const double *params, const double *x, int64_t batch,
                    double *out, double *acts) {
    for (int64_t r = 0; r < batch; ++r) {
        double cur[OR_GUIDE_IN], nxt[OR_GUIDE_IN];
        memcpy(cur, x + r * OR_GUIDE_IN, sizeof(double) * OR_GUIDE_IN);
        const double *W = params;
        for (int l = 0; l < 5; ++l) {
            int ni = g_dims[l], no = g_dims[l + 1];
            for (int o = 0; o < no; ++o) {
                double acc = 0.0;
                for (int i = 0; i < ni; ++i) acc += W[(size_t)o * ni + i] * cur[i];
                nxt[o] = (l < 4 && acc < 0.0) ? 0.0 : acc;
            }
            W += (size_t)ni * no;
            memcpy(cur, nxt, sizeof(double) * (size_t)no);
            if (acts && l < 4) memcpy(acts + (r * 4 + l) * OR_GUIDE_HID, cur, sizeof(double) * OR_GUIDE_HID);
        }
        memcpy(out + r * OR_GUIDE_OUT, cur, sizeof(double) * OR_GUIDE_OUT);
    }
}

static double softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }

void or_mixture_from_raw(const double *raw, double mu[8][3], double kappa[8],
                         double weight[8]) {
    double mx = -INFINITY;
    for (int k = 0; k < 8; ++k) mx = fmax(mx, raw[5 * k + 4]);
    double z = 0.0;
    for (int k = 0; k < 8; ++k) {
        const double *r = raw + 5 * k;
        double l = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (l > 0.0) { mu[k][0] = r[0] / l; mu[k][1] = r[1] / l; mu[k][2] = r[2] / l; }
        else { mu[k][0] = 0.0; mu[k][1] = 0.0; mu[k][2] = 1.0; }
        double kp = softplus(r[3]);
        kappa[k] = fmin(KMAX, fmax(KMIN, kp));
        weight[k] = exp(r[4] - mx);
        z += weight[k];
    }
    for (int k = 0; k < 8; ++k) weight[k] /= z;
}

double or_mixture_pdf(const double *raw, const double w[3]) {
    double mu[8][3], kp[8], wt[8];
    or_mixture_from_raw(raw, mu, kp, wt);
    double p = 0.0;
    for (int k = 0; k < 8; ++k) p += wt[k] * or_vmf_pdf(kp[k], mu[k], w);
    return p;
}

void or_mixture_sample(const double *raw, double u_sel, double u1, double u2,
                       double w[3]) {
    double mu[8][3], kp[8], wt[8];
    or_mixture_from_raw(raw, mu, kp, wt);
    int k = 0;
    double acc = 0.0;
    for (k = 0; k < 7; ++k) {
        if (u_sel < acc + wt[k]) break;
        acc += wt[k];
    }
    or_vmf_sample(kp[k], mu[k], u1, u2, w);
}

/* Loss and its gradient by backpropagation (double precision). */
double or_guide_loss_grad(const double *params, const double *x,
                          const double *wi, const double *weight,
                          int64_t batch, double *grad) {
    int64_t np = or_guide_nparams();
    memset(grad, 0, sizeof(double) * (size_t)np);
    double loss = 0.0;
    double *acts = (double *)malloc(sizeof(double) * 4 * OR_GUIDE_HID);
    for (int64_t r = 0; r < batch; ++r) {
        double raw[OR_GUIDE_OUT];
        or_mlp_forward(params, x + r * OR_GUIDE_IN, 1, raw, acts);
        double mu[8][3], kp[8], wt[8], q[8];
        or_mixture_from_raw(raw, mu, kp, wt);
        const double *w = wi + 3 * r;
        double qm = 0.0;
        for (int k = 0; k < 8; ++k) { q[k] = or_vmf_pdf(kp[k], mu[k], w); qm += wt[k] * q[k]; }
        double scale = weight[r] / (double)batch;
        loss += -scale * log(qm);
        /* d loss / d raw */
        double g[OR_GUIDE_OUT];
        for (int k = 0; k < 8; ++k) {
            const double *rk = raw + 5 * k;
            double resp = wt[k] * q[k] / qm;
            double c = mu[k][0] * w[0] + mu[k][1] * w[1] + mu[k][2] * w[2];
            double l = sqrt(rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2]);
            for (int a = 0; a < 3; ++a)
                g[5 * k + a] = l > 0.0 ? -scale * resp * kp[k] * (w[a] - c * mu[k][a]) / l : 0.0;
            double kpr = softplus(rk[3]);
            double dk = 0.0;
            if (kpr > KMIN && kpr < KMAX) {
                double dlogq = 1.0 / kp[k] - 2.0 / expm1(2.0 * kp[k]) + (c - 1.0);
                double sig = 1.0 / (1.0 + exp(-rk[3]));
                dk = resp * dlogq * sig;
            }
            g[5 * k + 3] = -scale * dk;
            g[5 * k + 4] = -scale * (resp - wt[k]);
        }
        /* backward through the layers */
        double dcur[OR_GUIDE_IN];
        memcpy(dcur, g, sizeof g);
        int64_t off[5]; int64_t o0 = 0;
        for (int l = 0; l < 5; ++l) { off[l] = o0; o0 += (int64_t)g_dims[l] * g_dims[l + 1]; }
        for (int l = 4; l >= 0; --l) {
            int ni = g_dims[l], no = g_dims[l + 1];
            const double *in = l == 0 ? x + r * OR_GUIDE_IN : acts + (l - 1) * OR_GUIDE_HID;
            const double *W = params + off[l];
            double *G = grad + off[l];
            for (int o = 0; o < no; ++o)
                for (int i = 0; i < ni; ++i) G[(size_t)o * ni + i] += dcur[o] * in[i];
            if (l == 0) break;
            double dprev[OR_GUIDE_IN];
            for (int i = 0; i < ni; ++i) {
                double acc = 0.0;
                for (int o = 0; o < no; ++o) acc += W[(size_t)o * ni + i] * dcur[o];
                dprev[i] = in[i] > 0.0 ? acc : 0.0; /* ReLU of layer l-1 */
            }
            memcpy(dcur, dprev, sizeof(double) * (size_t)ni);
        }
    }
    free(acts);
    return loss;
}

void or_adam_step(double *params, const double *grad, double *m, double *v,
                  int64_t n, int64_t t, double lr, double b1, double b2,
                  double eps) {
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        params[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
