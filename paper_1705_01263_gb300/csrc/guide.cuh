// Device-side math of the guiding proposal: one-blob input encoding, the
// 8-lobe von Mises-Fisher mixture decoded from the network outputs, its pdf
// and sampling, and the gradient of the training loss -w log q(wi) with
// respect to the raw outputs. Definitions (not from the paper, which has no
// learned component): vMF q(w) = k / (2 pi (1 - e^{-2k})) exp(k (mu.w - 1)),
// sampled as in Jakob 2012; one-blob bins per Mueller et al. 2019; mu =
// normalise(raw xyz), kappa = clamp(softplus(raw), 1e-2, 1e4), weights =
// softmax(logits).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace rtg {

constexpr int kGuideBins = 32;
constexpr int kGuideIn = 7 * kGuideBins;   // 224
constexpr int kGuideHid = 64;
constexpr int kGuideOut = 40;
constexpr int kGuideOutPad = 48;           // MMA N must be a multiple of 16
constexpr int kGuideLobes = 8;
constexpr int64_t kGuideParams = (int64_t)kGuideIn * kGuideHid + 3 * kGuideHid * kGuideHid + kGuideHid * kGuideOut;
constexpr float kKappaMin = 1e-2f, kKappaMax = 1e4f;

// One-blob bins c0 .. c0 + 7 (c0 a multiple of 8) of scalar s, the Gaussian
// exp(-(s - (c + 1/2) / 32)^2 / (2 sigma^2)) with sigma = 1/32: bin c0 by one
// exponential, its neighbours by the ratio of consecutive bins,
// g(c + 1) = g(c) r_c with r_c = exp(32 (s - (c + 1/2) / 32) - 1/2) and
// r_{c+1} = r_c / e (two exponentials per eight bins instead of eight).
RT_HD float oneblob_exp(float x) {
#ifdef __CUDA_ARCH__
    return __expf(x);   // the bins are rounded to BF16: the fast exponential's error is far below that
#else
    return expf(x);
#endif
}

RT_HD void oneblob_chunk(float s, int c0, float *g8) {
    const float sig = 1.f / kGuideBins;
    const float d = s - ((float)c0 + 0.5f) / kGuideBins;
    float g = oneblob_exp(-d * d / (2.f * sig * sig));
    float r = oneblob_exp((float)kGuideBins * d - 0.5f);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        g8[e] = g;
        g *= r;
        r *= 0.36787944117144233f;   // 1 / e
    }
}

RT_HD float oneblob_bin(float s, int c) {
    float g8[8];
    oneblob_chunk(s, c & ~7, g8);
    return g8[c & 7];
}

// Features in [0,1]: position in the scene box (3), outgoing direction and
// normal as ((cos theta + 1) / 2, phi / 2 pi) with theta measured from +y.
RT_HD void dir_features(V3 w, float &a, float &b) {
    float cy = fmaxf(-1.f, fminf(1.f, w.y));
    float phi = atan2f(w.z, w.x);
    if (phi < 0.f) phi += 2.f * kPi;
    a = 0.5f * (cy + 1.f);
    b = phi * (0.5f * kInvPi);
}

RT_HD void guide_features(V3 x, V3 wo, V3 n, float3 lo, float3 hi, float *f) {
    f[0] = fminf(1.f, fmaxf(0.f, (x.x - lo.x) / fmaxf(hi.x - lo.x, 1e-20f)));
    f[1] = fminf(1.f, fmaxf(0.f, (x.y - lo.y) / fmaxf(hi.y - lo.y, 1e-20f)));
    f[2] = fminf(1.f, fmaxf(0.f, (x.z - lo.z) / fmaxf(hi.z - lo.z, 1e-20f)));
    dir_features(wo, f[3], f[4]);
    dir_features(n, f[5], f[6]);
}

RT_HD float softplusf(float x) { return x > 20.f ? x : log1pf(expf(x)); }

// A decoded mixture: per lobe the mean direction mu (xyz), kappa, the
// weight w and c = w kappa / (2 pi (1 - e^{-2 kappa})), the weighted lobe's
// normalisation. Element (k, f) of lobe k, field f (0-2 mu, 3 kappa, 4 w,
// 5 c): Mixture keeps them in a thread-local array; MixtureStrided at
// p[(6 k + f) stride], so that a block's threads keep theirs in shared
// memory side by side (stride = threads of the block), out of the local
// memory that a thread-local array indexed by the sampled lobe lives in.
constexpr int kMixFields = 6;
struct Mixture {
    float v[kGuideLobes * kMixFields];
    RT_HD float &at(int k, int f) { return v[kMixFields * k + f]; }
    RT_HD float at(int k, int f) const { return v[kMixFields * k + f]; }
};
struct MixtureStrided {
    float *p;
    uint32_t stride;
    RT_HD float &at(int k, int f) const { return p[(size_t)(kMixFields * k + f) * stride]; }
};
template <class M>
RT_HD V3 mix_mu(const M &m, int k) { return v3(m.at(k, 0), m.at(k, 1), m.at(k, 2)); }
template <class M>
RT_HD float mix_kappa(const M &m, int k) { return m.at(k, 3); }
template <class M>
RT_HD float mix_w(const M &m, int k) { return m.at(k, 4); }
template <class M>
RT_HD float mix_c(const M &m, int k) { return m.at(k, 5); }

RT_HD float raw_value(float v) { return v; }
RT_HD float raw_value(__nv_bfloat16 v) { return __bfloat162float(v); }

// Raw outputs in FP32 (training, the API) or BF16 (the rows the guided
// render writes and reads back).
template <class T, class M>
RT_HD void decode_mixture(const T *raw, M &m) {
    float mx = -INFINITY;
    for (int k = 0; k < kGuideLobes; ++k) mx = fmaxf(mx, raw_value(raw[5 * k + 4]));
    float z = 0.f;
    for (int k = 0; k < kGuideLobes; ++k) {
        const T *rr = raw + 5 * k;
        const float r[4] = {raw_value(rr[0]), raw_value(rr[1]), raw_value(rr[2]), raw_value(rr[3])};
        const float l = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        const float il = l > 0.f ? 1.f / l : 0.f;
        const V3 mu = l > 0.f ? v3(r[0] * il, r[1] * il, r[2] * il) : v3(0.f, 0.f, 1.f);
        m.at(k, 0) = mu.x;
        m.at(k, 1) = mu.y;
        m.at(k, 2) = mu.z;
        m.at(k, 3) = fminf(kKappaMax, fmaxf(kKappaMin, softplusf(r[3])));
        const float w = expf(raw_value(rr[4]) - mx);
        m.at(k, 4) = w;
        z += w;
    }
    const float iz = 1.f / z;
    for (int k = 0; k < kGuideLobes; ++k) {
        const float w = m.at(k, 4) * iz, kap = m.at(k, 3);
        m.at(k, 4) = w;
        // 1 - e^{-2 kappa} rounds to 1 in FP32 once kappa > 9
        m.at(k, 5) = w * kap / (2.f * kPi * (kap > 9.f ? 1.f : -expm1f(-2.f * kap)));
    }
}

RT_HD float vmf_pdf(float kappa, V3 mu, V3 w) {
    return kappa / (2.f * kPi * -expm1f(-2.f * kappa)) * expf(kappa * (dot(mu, w) - 1.f));
}

template <class M>
RT_HD float mixture_pdf(const M &m, V3 w) {
    float p = 0.f;
    for (int k = 0; k < kGuideLobes; ++k) p += mix_c(m, k) * expf(mix_kappa(m, k) * (dot(mix_mu(m, k), w) - 1.f));
    return p;
}

// Lobe by u_sel, then cos theta = 1 + ln(u1 + (1 - u1) e^{-2k}) / k about mu.
template <class M>
RT_HD V3 mixture_sample(const M &m, float u_sel, float u1, float u2) {
    int k = 0;
    float acc = 0.f;
    for (k = 0; k < kGuideLobes - 1; ++k) {
        if (u_sel < acc + mix_w(m, k)) break;
        acc += mix_w(m, k);
    }
    const float kap = mix_kappa(m, k);
    const V3 n = mix_mu(m, k);
    float ct = 1.f + logf(u1 + (1.f - u1) * expf(-2.f * kap)) / kap;
    ct = fminf(1.f, fmaxf(-1.f, ct));
    float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
    float phi = 2.f * kPi * u2;
    float sign = n.z >= 0.f ? 1.f : -1.f;
    float a = -1.f / (sign + n.z);
    float bb = n.x * n.y * a;
    V3 t = v3(1.f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    V3 b = v3(bb, sign + n.y * n.y * a, -n.y);
    return normalize(st * cosf(phi) * t + st * sinf(phi) * b + ct * n);
}

// Loss contribution scale * -log q(wi) and its gradient w.r.t. raw (40
// entries written; entries 40..47 left untouched).
RT_HD float mixture_loss_grad(const float *raw, const float *wi3, float scale, float *g) {
    Mixture m;
    decode_mixture(raw, m);
    V3 wi = v3(wi3[0], wi3[1], wi3[2]);
    float q[kGuideLobes], qm = 0.f;
    for (int k = 0; k < kGuideLobes; ++k) {
        q[k] = vmf_pdf(mix_kappa(m, k), mix_mu(m, k), wi);
        qm += mix_w(m, k) * q[k];
    }
    qm = fmaxf(qm, 1e-30f);
    for (int k = 0; k < kGuideLobes; ++k) {
        const float *rk = raw + 5 * k;
        float resp = mix_w(m, k) * q[k] / qm;
        const V3 mu = mix_mu(m, k);
        const float kk = mix_kappa(m, k);
        float c = dot(mu, wi);
        float l = sqrtf(rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2]);
        float inv_l = l > 0.f ? 1.f / l : 0.f;
        g[5 * k + 0] = -scale * resp * kk * (wi.x - c * mu.x) * inv_l;
        g[5 * k + 1] = -scale * resp * kk * (wi.y - c * mu.y) * inv_l;
        g[5 * k + 2] = -scale * resp * kk * (wi.z - c * mu.z) * inv_l;
        float sp = softplusf(rk[3]);
        float dk = 0.f;
        if (sp > kKappaMin && sp < kKappaMax) {
            float dlogq = 1.f / kk - 2.f / expm1f(2.f * kk) + (c - 1.f);
            dk = resp * dlogq / (1.f + expf(-rk[3]));
        }
        g[5 * k + 3] = -scale * dk;
        g[5 * k + 4] = -scale * (resp - mix_w(m, k));
    }
    return -scale * logf(qm);
}

}  // namespace rtg
