// Photon aiming (paper Sec. 2.1.3): the light-tracing stage picks a cluster
// of objects by descending the cluster hierarchy (DevScene::pa_node /
// pa_link), each step choosing a child in proportion to an optimistic
// estimate of the screen-space photon density it would receive, and aims the
// photon uniformly at that cluster's sphere. The density of an emission for
// MIS is summed over every cluster whose sphere the emission ray passes,
// found by traversing the same hierarchy with the ray.
//
// Estimate of a node (the optimistic bound the paper asks for): the solid
// angle 2 pi (1 - sqrt(1 - r^2/d^2)) under which the eye sees the node's
// sphere, 4 pi when the eye is inside, at most the solid angle of the
// camera's view cone (the cone around the optical axis through the image
// corners): no cluster takes more than the whole screen. A photon aimed
// uniformly at a sphere of radius r lays 1 / (pi r^2) photons per unit area
// across it and a pixel at distance d covers an area proportional to d^2,
// so clusters chosen in proportion to their solid angle receive about as
// many photons per pixel; the cap keeps a cluster around the eye (a ground)
// from taking photons that its huge sphere mostly sends out of view. For a
// photon from a triangle emitter (point y, normal ny) a node whose sphere
// lies wholly behind the emitter's plane gets zero (the emitter radiates on
// its normal's side only). `eye` = (position, view-cone solid angle).
#pragma once

#include "common.cuh"

namespace rtg {

constexpr int kAimStack = 48;   // traversal stack: the hierarchy is a median split, depth <= log2(clusters) + 1

RT_HD float aim_estimate(float4 sph, float4 eye, bool from_tri, V3 y, V3 ny) {
    const V3 c = v3(sph.x, sph.y, sph.z);
    if (from_tri && !(dot(c - y, ny) > -sph.w)) return 0.f;
    const V3 v = c - v3(eye.x, eye.y, eye.z);
    const float d2 = dot(v, v), r2 = sph.w * sph.w;
    float om = 4.f * kPi;
    if (d2 > r2) {
        const float x = r2 / d2;
        om = 2.f * kPi * x / (1.f + sqrtf(1.f - x));   // 2 pi (1 - sqrt(1 - x)), without cancellation
    }
    return fminf(om, eye.w);
}

RT_HD float aim_p_left(const DevScene &sc, int2 link, float4 eye, bool from_tri, V3 y, V3 ny) {
    const float wl = aim_estimate(ldg(sc.pa_node + link.x), eye, from_tri, y, ny);
    const float wr = aim_estimate(ldg(sc.pa_node + link.y), eye, from_tri, y, ny);
    if (!(wl + wr > 0.f)) return 0.5f;
    return wl / (wl + wr);
}

// Descent driven by one uniform number (rescaled at each level); returns the
// chosen cluster's sphere.
RT_HD float4 aim_sample(const DevScene &sc, float4 eye, bool from_tri, V3 y, V3 ny, float u) {
    int node = 0;
    for (;;) {
        const int2 link = ldg(sc.pa_link + node);
        if (link.x < 0) return ldg(sc.pa_node + node);
        const float pl = aim_p_left(sc, link, eye, from_tri, y, ny);
        if (u < pl) {
            u = u / pl;
            node = link.x;
        } else {
            u = (u - pl) / (1.f - pl);
            node = link.y;
        }
        u = fminf(u, 0.99999994f);
    }
}

// Line through x along unit w meets the sphere: the centre's distance to
// the line, |v x w| (no cancellation, unlike |v|^2 - (v.w)^2 in FP32 far
// from the sphere), at most the radius.
RT_HD bool aim_line_meets(float4 sph, V3 x, V3 w) {
    const V3 q = cross(v3(sph.x, sph.y, sph.z) - x, w);
    return dot(q, q) <= sph.w * sph.w;
}

// Ray from y along unit w passes through the sphere: y inside it, or the
// centre ahead and within the radius of the ray's line (the same as w inside
// the cone the sphere subtends from y, without comparing two cosines near 1).
RT_HD bool aim_cone_holds(float4 sph, V3 y, V3 w) {
    const V3 v = v3(sph.x, sph.y, sph.z) - y;
    const float r2 = sph.w * sph.w;
    if (dot(v, v) <= r2) return true;
    const V3 q = cross(v, w);
    return dot(v, w) > 0.f && dot(q, q) <= r2;
}

// Environment photon: density per unit area across w of the photon line
// through x, sum over clusters whose sphere the line meets of P_c / (pi r^2).
RT_HD float aim_env_density(const DevScene &sc, float4 eye, V3 x, V3 w) {
    if (sc.pa_nnodes <= 0) return 0.f;
    int stack[kAimStack];
    float pstack[kAimStack];
    int sp = 0;
    stack[sp] = 0;
    pstack[sp++] = 1.f;
    float sum = 0.f;
    while (sp > 0) {
        --sp;
        const int node = stack[sp];
        const float p = pstack[sp];
        const float4 sph = ldg(sc.pa_node + node);
        if (!(p > 0.f) || !aim_line_meets(sph, x, w)) continue;
        const int2 link = ldg(sc.pa_link + node);
        if (link.x < 0) {
            sum += p / (kPi * sph.w * sph.w);
            continue;
        }
        if (sp + 2 > kAimStack) break;
        const float pl = aim_p_left(sc, link, eye, false, x, w);
        stack[sp] = link.y; pstack[sp++] = p * (1.f - pl);
        stack[sp] = link.x; pstack[sp++] = p * pl;
    }
    return sum;
}

// Triangle photon from y (emitter normal ny) leaving along w: solid-angle
// density, sum over clusters whose cone holds w of P_c(y) / (2 pi (1 - cos
// theta_c)), or P_c(y) / (4 pi) when y is inside the cluster's sphere.
RT_HD float aim_dir_density(const DevScene &sc, float4 eye, V3 y, V3 ny, V3 w) {
    if (sc.pa_nnodes <= 0) return 0.f;
    int stack[kAimStack];
    float pstack[kAimStack];
    int sp = 0;
    stack[sp] = 0;
    pstack[sp++] = 1.f;
    float sum = 0.f;
    while (sp > 0) {
        --sp;
        const int node = stack[sp];
        const float p = pstack[sp];
        const float4 sph = ldg(sc.pa_node + node);
        if (!(p > 0.f) || !aim_cone_holds(sph, y, w)) continue;
        const int2 link = ldg(sc.pa_link + node);
        if (link.x < 0) {
            const V3 v = v3(sph.x, sph.y, sph.z) - y;
            const float d2 = dot(v, v), r2 = sph.w * sph.w;
            if (d2 <= r2) {
                sum += p / (4.f * kPi);
            } else {
                const float x = r2 / d2;
                sum += p * (1.f + sqrtf(1.f - x)) / (2.f * kPi * x);   // p / (2 pi (1 - cos theta_max))
            }
            continue;
        }
        if (sp + 2 > kAimStack) break;
        const float pl = aim_p_left(sc, link, eye, true, y, ny);
        stack[sp] = link.y; pstack[sp++] = p * (1.f - pl);
        stack[sp] = link.x; pstack[sp++] = p * pl;
    }
    return sum;
}

// Direction uniform in the cone from y subtending the sphere (uniform over
// all directions when y is inside it).
RT_HD V3 aim_cone_sample(float4 sph, V3 y, float u1, float u2) {
    V3 axis = v3(0.f, 0.f, 1.f);
    const V3 v = v3(sph.x, sph.y, sph.z) - y;
    const float d2 = dot(v, v), r2 = sph.w * sph.w;
    float ct;
    if (d2 <= r2) {
        ct = 1.f - 2.f * u1;
    } else {
        axis = v * (1.f / sqrtf(d2));
        const float x = r2 / d2;
        ct = 1.f - u1 * (x / (1.f + sqrtf(1.f - x)));
    }
    const float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
    const float s = sinf(2.f * kPi * u2), c = cosf(2.f * kPi * u2);
    V3 t1, t2;
    onb(axis, t1, t2);
    return normalize((st * c) * t1 + (st * s) * t2 + ct * axis);
}

}  // namespace rtg
