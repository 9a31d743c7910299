/*
 * Oracle: local shading in FP64 (paper Sec. 2.2 stage 1 "state setup" and
 * stage 4 "evaluation and sampling of the layered BSDF"; Appendix A.3 "local
 * shading normal adaptation").
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper names a generic layered BSDF but prints no formula; the material
 * used here is the reading fixed for the synthetic scenes: a mixture
 *     f = w * f_ggx + (1 - w) * albedo / pi
 * with f_ggx the isotropic GGX microfacet reflection of Walter et al. 2007
 * (alpha = roughness^2, height-correlated Smith masking-shadowing of Heitz
 * 2014, Schlick Fresnel with F0 = 0.04), sampled by choosing a lobe with
 * probability w, the GGX lobe by visible-normal sampling (Heitz, JCGT 2018)
 * and the diffuse lobe by cosine-weighted sampling; the returned pdf is
 * always the full mixture pdf.
 */
#include "oracle.h"
#include <math.h>

#define OR_PI 3.14159265358979323846
#define OR_F0 0.04
#define OR_ADAPT_EPS 1e-3

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void normalize3(double a[3]) {
    double l = sqrt(dot3(a, a));
    if (l > 0.0) { a[0] /= l; a[1] /= l; a[2] /= l; }
}

double or_luminance(const double c[3]) {
    return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2];
}

/* Orthonormal basis around unit n (Duff et al., JCGT 2017). */
void or_onb(const double n[3], double t[3], double b[3]) {
    double sign = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sign + n[2]);
    double bb = n[0] * n[1] * a;
    t[0] = 1.0 + sign * n[0] * n[0] * a; t[1] = sign * bb; t[2] = -sign * n[0];
    b[0] = bb; b[1] = sign + n[1] * n[1] * a; b[2] = -n[1];
}

/* Appendix A.3. ns and ng are unit, ng faces wo (dot(wo, ng) > 0) and ns
 * lies on ng's side. Reflect wo about ns; if the reflection is not at least
 * OR_ADAPT_EPS above the geometric tangent plane, add t*ng with t chosen in
 * closed form so that the normalized result has dot(r', ng) == OR_ADAPT_EPS,
 * and return the half vector of wo and r'. */
void or_adapt_shading_normal(const double ns[3], const double ng[3],
                             const double wo[3], double out[3]) {
    double c = dot3(wo, ns);
    double r[3] = {2.0 * c * ns[0] - wo[0], 2.0 * c * ns[1] - wo[1], 2.0 * c * ns[2] - wo[2]};
    double a = dot3(r, ng);
    if (a >= OR_ADAPT_EPS) { out[0] = ns[0]; out[1] = ns[1]; out[2] = ns[2]; return; }
    double e = OR_ADAPT_EPS;
    double s = e * sqrt(fmax(0.0, (1.0 - a * a) / (1.0 - e * e)));
    double t = s - a;
    double rp[3] = {r[0] + t * ng[0], r[1] + t * ng[1], r[2] + t * ng[2]};
    double lr = sqrt(dot3(rp, rp));
    if (!(lr > 1e-12)) { out[0] = ng[0]; out[1] = ng[1]; out[2] = ng[2]; return; }
    rp[0] /= lr; rp[1] /= lr; rp[2] /= lr;
    double h[3] = {wo[0] + rp[0], wo[1] + rp[1], wo[2] + rp[2]};
    double lh = sqrt(dot3(h, h));
    if (!(lh > 1e-12)) { out[0] = ng[0]; out[1] = ng[1]; out[2] = ng[2]; return; }
    out[0] = h[0] / lh; out[1] = h[1] / lh; out[2] = h[2] / lh;
}

double or_ggx_D(double alpha, double cos_h) {
    if (cos_h <= 0.0) return 0.0;
    double a2 = alpha * alpha;
    double k = cos_h * cos_h * (a2 - 1.0) + 1.0;
    return a2 / (OR_PI * k * k);
}

double or_ggx_lambda(double alpha, double cos_t) {
    double c2 = cos_t * cos_t;
    double tan2 = fmax(0.0, 1.0 - c2) / c2;
    return 0.5 * (-1.0 + sqrt(1.0 + alpha * alpha * tan2));
}

double or_ggx_G1(double alpha, double cos_t) {
    return 1.0 / (1.0 + or_ggx_lambda(alpha, cos_t));
}

double or_schlick(double cos_ih) {
    double m = 1.0 - fmax(0.0, fmin(1.0, cos_ih));
    double m2 = m * m;
    return OR_F0 + (1.0 - OR_F0) * m2 * m2 * m;
}

static double ggx_alpha(double rough) {
    double a = rough * rough;
    return a < 1e-4 ? 1e-4 : a;
}

void or_bsdf_eval(const double albedo[3], double rough, double w,
                  const double ns[3], const double wo[3], const double wi[3],
                  double f[3], double *pdf) {
    double co = dot3(wo, ns), ci = dot3(wi, ns);
    f[0] = f[1] = f[2] = 0.0; *pdf = 0.0;
    if (co <= 0.0 || ci <= 0.0) return;
    double alpha = ggx_alpha(rough);
    double h[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    normalize3(h);
    double ch = dot3(h, ns), cih = dot3(wi, h);
    double D = or_ggx_D(alpha, ch);
    double G2 = 1.0 / (1.0 + or_ggx_lambda(alpha, co) + or_ggx_lambda(alpha, ci));
    double F = or_schlick(cih);
    double spec = D * G2 * F / (4.0 * co * ci);
    for (int c = 0; c < 3; ++c) f[c] = w * spec + (1.0 - w) * albedo[c] / OR_PI;
    double pdf_spec = or_ggx_G1(alpha, co) * D / (4.0 * co);
    double pdf_diff = ci / OR_PI;
    *pdf = w * pdf_spec + (1.0 - w) * pdf_diff;
}

/* Visible-normal sampling of GGX, in the local frame (z = normal). */
void or_ggx_vndf_sample(double alpha, const double v[3], double u1, double u2,
                        double h[3]) {
    double vh[3] = {alpha * v[0], alpha * v[1], v[2]};
    normalize3(vh);
    double lensq = vh[0] * vh[0] + vh[1] * vh[1];
    double T1[3];
    if (lensq > 0.0) {
        double il = 1.0 / sqrt(lensq);
        T1[0] = -vh[1] * il; T1[1] = vh[0] * il; T1[2] = 0.0;
    } else { T1[0] = 1.0; T1[1] = 0.0; T1[2] = 0.0; }
    double T2[3] = {vh[1] * T1[2] - vh[2] * T1[1], vh[2] * T1[0] - vh[0] * T1[2],
                    vh[0] * T1[1] - vh[1] * T1[0]};
    double r = sqrt(u1), phi = 2.0 * OR_PI * u2;
    double t1 = r * cos(phi), t2 = r * sin(phi);
    double s = 0.5 * (1.0 + vh[2]);
    t2 = (1.0 - s) * sqrt(fmax(0.0, 1.0 - t1 * t1)) + s * t2;
    double tz = sqrt(fmax(0.0, 1.0 - t1 * t1 - t2 * t2));
    double nh[3];
    for (int a = 0; a < 3; ++a) nh[a] = t1 * T1[a] + t2 * T2[a] + tz * vh[a];
    h[0] = alpha * nh[0]; h[1] = alpha * nh[1]; h[2] = fmax(0.0, nh[2]);
    normalize3(h);
}

int or_bsdf_sample(const double albedo[3], double rough, double w,
                   const double ns[3], const double wo[3], double u_lobe,
                   double u1, double u2, double wi[3], double f[3],
                   double *pdf) {
    double t[3], b[3];
    or_onb(ns, t, b);
    double co = dot3(wo, ns);
    *pdf = 0.0; f[0] = f[1] = f[2] = 0.0;
    if (co <= 0.0) return 0;
    double local[3];
    if (u_lobe < w) {
        double vl[3] = {dot3(wo, t), dot3(wo, b), co};
        double h[3];
        or_ggx_vndf_sample(ggx_alpha(rough), vl, u1, u2, h);
        double vh = dot3(vl, h);
        for (int a = 0; a < 3; ++a) local[a] = 2.0 * vh * h[a] - vl[a];
    } else {
        double r = sqrt(u1), phi = 2.0 * OR_PI * u2;
        local[0] = r * cos(phi); local[1] = r * sin(phi);
        local[2] = sqrt(fmax(0.0, 1.0 - u1));
    }
    for (int a = 0; a < 3; ++a)
        wi[a] = local[0] * t[a] + local[1] * b[a] + local[2] * ns[a];
    normalize3(wi);
    or_bsdf_eval(albedo, rough, w, ns, wo, wi, f, pdf);
    return *pdf > 0.0;
}
