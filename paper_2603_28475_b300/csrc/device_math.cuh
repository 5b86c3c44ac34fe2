// Device arithmetic of the PNCG-IPC solve: Neo-Hookean per-tet terms in a
// small-strain-stable float32 form, contact distances with their first and
// second directional derivatives in float64, barrier and friction terms.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace tac {

// ---------------------------------------------------------------------------
// Neo-Hookean, Psi(F) = mu/2 (|F|^2 - 3) - mu ln J + lam/2 (ln J)^2 (Supp. A).
// All quantities are formed from the displacement gradient G = F - I so that
// nothing cancels against the identity: J - 1 = tr G + i2(G) + det G,
// cof(F) = (1 + tr G) I - G^T + cof(G), and
// J F - cof(F) = G + G^T + (i2 + det G) I + (J - 1) G - cof(G).

struct FAnalysis {
    float cof[9];   // cof(F) (row-major), F^-T = cof / J
    float J, lnJ, invJ;
    float Q[9];     // J F - cof(F)
};

__device__ __forceinline__ void f_analysis(const float G[9], FAnalysis& f) {
    float cg0 = G[4] * G[8] - G[5] * G[7];
    float cg1 = G[5] * G[6] - G[3] * G[8];
    float cg2 = G[3] * G[7] - G[4] * G[6];
    float cg3 = G[2] * G[7] - G[1] * G[8];
    float cg4 = G[0] * G[8] - G[2] * G[6];
    float cg5 = G[1] * G[6] - G[0] * G[7];
    float cg6 = G[1] * G[5] - G[2] * G[4];
    float cg7 = G[2] * G[3] - G[0] * G[5];
    float cg8 = G[0] * G[4] - G[1] * G[3];
    float trG = G[0] + G[4] + G[8];
    float i2 = cg0 + cg4 + cg8;
    float detG = G[0] * cg0 + G[1] * cg1 + G[2] * cg2;
    float a = trG + (i2 + detG);
    f.J = 1.0f + a;
    f.lnJ = log1pf(a);
    f.invJ = 1.0f / f.J;
    float d = 1.0f + trG;
    f.cof[0] = cg0 - G[0] + d; f.cof[1] = cg1 - G[3];     f.cof[2] = cg2 - G[6];
    f.cof[3] = cg3 - G[1];     f.cof[4] = cg4 - G[4] + d; f.cof[5] = cg5 - G[7];
    f.cof[6] = cg6 - G[2];     f.cof[7] = cg7 - G[5];     f.cof[8] = cg8 - G[8] + d;
    float s2 = i2 + detG;
    f.Q[0] = 2.0f * G[0] + s2 + a * G[0] - cg0;
    f.Q[4] = 2.0f * G[4] + s2 + a * G[4] - cg4;
    f.Q[8] = 2.0f * G[8] + s2 + a * G[8] - cg8;
    f.Q[1] = G[1] + G[3] + a * G[1] - cg1;
    f.Q[3] = G[3] + G[1] + a * G[3] - cg3;
    f.Q[2] = G[2] + G[6] + a * G[2] - cg2;
    f.Q[6] = G[6] + G[2] + a * G[6] - cg6;
    f.Q[5] = G[5] + G[7] + a * G[5] - cg5;
    f.Q[7] = G[7] + G[5] + a * G[7] - cg7;
}

// ln(1 + q) - q, accurate for small q (series below 1e-2).
__device__ __forceinline__ float log1p_minus(float q) {
    if (fabsf(q) < 1e-2f) {
        float q2 = q * q;
        return q2 * (-0.5f + q * (1.0f / 3.0f + q * (-0.25f + q * 0.2f)));
    }
    return log1pf(q) - q;
}

// A = F^-1 dF = cof(F)^T dF / J; returns tr A, tr(A^2) and the invariants
// of A needed by the line remainder.
struct AInv {
    float c1, c2, c3, trA2;
};

__device__ __forceinline__ AInv a_invariants(const FAnalysis& f, const float dF[9]) {
    float A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            A[3 * i + j] = (f.cof[i] * dF[j] + f.cof[3 + i] * dF[3 + j] + f.cof[6 + i] * dF[6 + j]) * f.invJ;
    AInv r;
    r.c1 = A[0] + A[4] + A[8];
    float m0 = A[4] * A[8] - A[5] * A[7];
    float m4 = A[0] * A[8] - A[2] * A[6];
    float m8 = A[0] * A[4] - A[1] * A[3];
    r.c2 = m0 + m4 + m8;
    r.c3 = A[0] * m0 - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
    r.trA2 = A[0] * A[0] + A[4] * A[4] + A[8] * A[8] + 2.0f * (A[1] * A[3] + A[2] * A[6] + A[5] * A[7]);
    return r;
}

// ---------------------------------------------------------------------------
// Barrier b(d) = -(d - dhat)^2 ln(d / dhat) on 0 < d < dhat (Eq. ipc_energy).

__device__ __forceinline__ double barrier_b(double d, double dh) {
    if (d >= dh) return 0.0;
    double t = d - dh;
    return -t * t * log(d / dh);
}
__device__ __forceinline__ double barrier_b1(double d, double dh) {
    if (d >= dh) return 0.0;
    double t = d - dh;
    return -2.0 * t * log(d / dh) - t * t / d;
}
__device__ __forceinline__ double barrier_b2(double d, double dh) {
    if (d >= dh) return 0.0;
    double t = d - dh;
    return -2.0 * log(d / dh) - 4.0 * t / d + t * t / (d * d);
}

// b, b' and b'' together from one logarithm and one reciprocal (float64 is a
// narrow pipe; the three separate forms above cost three of each). T =
// float is the plain-FP32 form's barrier.
template <typename T>
struct Barrier3T {
    T b, b1, b2;
};
using Barrier3 = Barrier3T<double>;
template <typename T>
__device__ __forceinline__ Barrier3T<T> barrier_all(T d, T dh) {
    if (d >= dh) return Barrier3T<T>{T(0), T(0), T(0)};
    const T t = d - dh, L = log(d / dh), id = T(1) / d;
    const T ti = t * id;
    return Barrier3T<T>{-t * t * L, T(-2) * t * L - t * ti, T(-2) * L - T(4) * ti + ti * ti};
}

// ---------------------------------------------------------------------------
// Contact features. A pair has 4 slots; r = sum_s w_s v_s is the vector
// between the closest points (indenter -> gel), d = |r|. Within the active
// feature the weights are affine in nf free parameters theta:
// w = w0 + sum_k theta_k e_k, which gives the directional derivatives.

template <typename T>
struct V3 {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> v3(T a, T b, T c) { return V3<T>{a, b, c}; }
template <typename T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

template <typename T>
struct Feature {
    T d;
    T w[4];
    T e[2][4];
    int nf;
};

template <typename T>
__device__ __forceinline__ T clamp01(T t) { return t < T(0) ? T(0) : (t > T(1) ? T(1) : t); }

// point P vs segment AB: squared distance and parameter t (Q = A + t (B - A))
template <typename T>
__device__ __forceinline__ T seg_param(V3<T> P, V3<T> A, V3<T> B, T& t) {
    V3<T> e = B - A;
    T ee = dot(e, e);
    t = ee > T(0) ? clamp01(dot(P - A, e) / ee) : T(0);
    V3<T> r = P - (A + t * e);
    return dot(r, r);
}

// Point-triangle feature with slots [P, A, B, C], r = P - closest.
// Candidates: face interior (if the projection is inside), then edges AB,
// BC, CA with clamped parameters; the first minimum wins. Bit c of mask
// selects candidate c (0 face, 1 AB, 2 BC, 3 CA); a candidate left out must
// be known to lose, which pt_mask certifies from a float32 evaluation. The
// candidates evaluated are computed exactly as in the full search, so a
// certified mask gives the full search's result bit for bit.
template <typename T>
__device__ Feature<T> pt_feature(V3<T> P, V3<T> A, V3<T> B, V3<T> C, int mask = 15) {
    Feature<T> f;
    T best = sizeof(T) == 8 ? T(1e300) : T(3e38);
    int k = -1;
    T l0 = T(0), l1 = T(0), l2 = T(0), tab = T(0), tbc = T(0), tca = T(0);
    if (mask & 1) {
        V3<T> v0 = B - A, v1 = C - A, v2 = P - A;
        T d00 = dot(v0, v0), d01 = dot(v0, v1), d11 = dot(v1, v1), d20 = dot(v2, v0), d21 = dot(v2, v1);
        T den = d00 * d11 - d01 * d01;
        l1 = (d11 * d20 - d01 * d21) / den;
        l2 = (d00 * d21 - d01 * d20) / den;
        l0 = T(1) - l1 - l2;
        if (l0 >= T(0) && l1 >= T(0) && l2 >= T(0) && den > T(0)) {
            V3<T> n = cross(v0, v1);
            T s = dot(v2, n);
            best = s * s / dot(n, n);
            k = 0;
        }
    }
    if (k < 0 && !(mask & 14)) mask |= 14;   // the face alone was certified and failed: every edge
    if (mask & 2) {
        T dab = seg_param(P, A, B, tab);
        if (k < 0 || dab < best) { best = dab; k = 1; }
    }
    if (mask & 4) {
        T dbc = seg_param(P, B, C, tbc);
        if (k < 0 || dbc < best) { best = dbc; k = 2; }
    }
    if (mask & 8) {
        T dca = seg_param(P, C, A, tca);
        if (k < 0 || dca < best) { best = dca; k = 3; }
    }
    f.d = sqrt(best);
    f.nf = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) f.e[0][i] = f.e[1][i] = T(0);
    f.w[0] = T(1);
    if (k == 0) {
        f.w[1] = -l0; f.w[2] = -l1; f.w[3] = -l2;
        f.nf = 2;
        f.e[0][1] = T(1); f.e[0][2] = T(-1);
        f.e[1][1] = T(1); f.e[1][3] = T(-1);
    } else if (k == 1) {
        f.w[1] = -(T(1) - tab); f.w[2] = -tab; f.w[3] = T(0);
        if (tab > T(0) && tab < T(1)) { f.nf = 1; f.e[0][1] = T(1); f.e[0][2] = T(-1); }
    } else if (k == 2) {
        f.w[1] = T(0); f.w[2] = -(T(1) - tbc); f.w[3] = -tbc;
        if (tbc > T(0) && tbc < T(1)) { f.nf = 1; f.e[0][2] = T(1); f.e[0][3] = T(-1); }
    } else {
        f.w[1] = -tca; f.w[2] = T(0); f.w[3] = -(T(1) - tca);
        if (tca > T(0) && tca < T(1)) { f.nf = 1; f.e[0][3] = T(1); f.e[0][1] = T(-1); }
    }
    return f;
}

// Segment-segment feature with slots [P0, P1, Q0, Q1], r = P(s) - Q(t).
// Candidates: both interior (non-parallel, unconstrained solution inside
// [0,1]^2), then P0-vs-Q, P1-vs-Q, Q0-vs-P, Q1-vs-P; the first minimum wins.
// Bit c of mask selects candidate c, as for pt_feature (ee_mask certifies).
template <typename T>
__device__ Feature<T> ee_feature(V3<T> P0, V3<T> P1, V3<T> Q0, V3<T> Q1, int mask = 31) {
    Feature<T> f;
    T best = sizeof(T) == 8 ? T(1e300) : T(3e38);
    int k = -1;
    T s = T(0), t = T(0);
    if (mask & 1) {
        V3<T> u = P1 - P0, v = Q1 - Q0, w = P0 - Q0;
        T a = dot(u, u), b = dot(u, v), c = dot(v, v), dd = dot(u, w), e = dot(v, w);
        T D = a * c - b * b;
        if (D > T(1e-12) * a * c) {
            s = (b * e - c * dd) / D;
            t = (a * e - b * dd) / D;
            if (s >= T(0) && s <= T(1) && t >= T(0) && t <= T(1)) {
                V3<T> r = w + s * u - t * v;
                best = dot(r, r);
                k = 0;
            }
        }
    }
    if (k < 0 && !(mask & 30)) mask |= 30;   // the interior alone was certified and failed
    T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
    if (mask & 2) {
        T d0 = seg_param(P0, Q0, Q1, t0);
        if (k < 0 || d0 < best) { best = d0; k = 1; }
    }
    if (mask & 4) {
        T d1 = seg_param(P1, Q0, Q1, t1);
        if (k < 0 || d1 < best) { best = d1; k = 2; }
    }
    if (mask & 8) {
        T d2 = seg_param(Q0, P0, P1, t2);
        if (k < 0 || d2 < best) { best = d2; k = 3; }
    }
    if (mask & 16) {
        T d3 = seg_param(Q1, P0, P1, t3);
        if (k < 0 || d3 < best) { best = d3; k = 4; }
    }
    f.d = sqrt(best);
#pragma unroll
    for (int i = 0; i < 4; ++i) f.e[0][i] = f.e[1][i] = T(0);
    f.nf = 0;
    T sp, tq;
    bool sfree = false, tfree = false;
    if (k == 0) { sp = s; tq = t; sfree = tfree = true; }
    else if (k == 1) { sp = T(0); tq = t0; tfree = t0 > T(0) && t0 < T(1); }
    else if (k == 2) { sp = T(1); tq = t1; tfree = t1 > T(0) && t1 < T(1); }
    else if (k == 3) { sp = t2; tq = T(0); sfree = t2 > T(0) && t2 < T(1); }
    else { sp = t3; tq = T(1); sfree = t3 > T(0) && t3 < T(1); }
    f.w[0] = T(1) - sp; f.w[1] = sp; f.w[2] = -(T(1) - tq); f.w[3] = -tq;
    if (sfree) { f.e[f.nf][0] = T(-1); f.e[f.nf][1] = T(1); f.nf++; }
    if (tfree) { f.e[f.nf][2] = T(1); f.e[f.nf][3] = T(-1); f.nf++; }
    return f;
}

// ---------------------------------------------------------------------------
// Float32 certification of the closest-feature search. The float32 slot
// positions differ from the float64 ones by at most ex per coordinate, so a
// point-segment candidate's float32 distance is within err = 6 ex + 2^-20 d
// of its float64 value (the distance is 1-Lipschitz in each slot; the
// clamped parameter's own error is second order). A candidate whose float32
// distance exceeds the best by more than 2 err cannot win the float64
// search. The face (point-triangle) and the interior (edge-edge) candidate,
// when their projection lies inside with a margin, are the exact minimum
// and win alone; within the margin the float64 search decides. The masks
// keep every candidate that can win, so the float64 search over them
// returns what the full search returns.

__device__ __forceinline__ float cert_err(float ex, float d) { return 6.0f * ex + 9.5367431640625e-7f * d; }

// point-triangle, slots [P, A, B, C]; dmin as pt_feature<float>
__device__ __forceinline__ int pt_mask(V3<float> P, V3<float> A, V3<float> B, V3<float> C, float ex, float& dmin) {
    V3<float> v0 = B - A, v1 = C - A, v2 = P - A;
    float d00 = dot(v0, v0), d01 = dot(v0, v1), d11 = dot(v1, v1), d20 = dot(v2, v0), d21 = dot(v2, v1);
    float den = d00 * d11 - d01 * d01;
    float l1 = (d11 * d20 - d01 * d21) / den;
    float l2 = (d00 * d21 - d01 * d20) / den;
    float l0 = 1.0f - l1 - l2;
    float best = 3e38f;
    if (l0 >= 0.0f && l1 >= 0.0f && l2 >= 0.0f && den > 0.0f) {
        V3<float> n = cross(v0, v1);
        float s = dot(v2, n);
        best = s * s / dot(n, n);
    }
    // face status from the projection's distance to each edge line,
    // l_i |n| / |edge opposite i|: 1 inside, 0 outside, -1 within 16 ex
    int face = -1;
    if (den > 1e-6f * d00 * d11) {
        const float nn = sqrtf(den), tol = 16.0f * ex;
        const V3<float> v3 = v1 - v0;
        const float m0 = l0 * nn / sqrtf(dot(v3, v3)), m1 = l1 * nn / sqrtf(d11), m2 = l2 * nn / sqrtf(d00);
        if (m0 >= tol && m1 >= tol && m2 >= tol) face = 1;
        else if (m0 <= -tol || m1 <= -tol || m2 <= -tol) face = 0;
    }
    float t;
    const float de[3] = {seg_param(P, A, B, t), seg_param(P, B, C, t), seg_param(P, C, A, t)};
    float emin = fminf(de[0], fminf(de[1], de[2]));
    if (best > 2.9e38f || emin < best) best = emin;
    dmin = sqrtf(best);
    if (face == 1) return 1;
    const float r = sqrtf(emin), lim = r + 2.0f * cert_err(ex, r), lim2 = lim * lim;
    int mask = face < 0 ? 1 : 0;
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (de[j] <= lim2) mask |= 2 << j;
    return mask;
}

// edge-edge, slots [P0, P1, Q0, Q1]; dmin as ee_feature<float>
__device__ __forceinline__ int ee_mask(V3<float> P0, V3<float> P1, V3<float> Q0, V3<float> Q1, float ex, float& dmin) {
    V3<float> u = P1 - P0, v = Q1 - Q0, w = P0 - Q0;
    float a = dot(u, u), b = dot(u, v), c = dot(v, v), dd = dot(u, w), e = dot(v, w);
    float D = a * c - b * b;
    float best = 3e38f;
    int inter = -1;   // 1 interior inside, 0 outside, -1 uncertain
    if (D > 1e-12f * a * c) {
        float s = (b * e - c * dd) / D;
        float t = (a * e - b * dd) / D;
        if (s >= 0.0f && s <= 1.0f && t >= 0.0f && t <= 1.0f) {
            V3<float> r = w + s * u - t * v;
            best = dot(r, r);
        }
        if (D > 1e-4f * a * c) {
            // the closest points move by ex / sin(angle) along the edges;
            // the float32 solve loses (a c / D) ulps to cancellation
            const float iD = 1.0f / D, sD = sqrtf(D), cond = a * c * iD;
            const float ar = 1.9073486328125e-6f * cond * (1.0f + sqrtf(dot(w, w) / fminf(a, c)));
            const float ms = 16.0f * ex * sqrtf(c) / sD + ar, mt = 16.0f * ex * sqrtf(a) / sD + ar;
            if (s >= ms && s <= 1.0f - ms && t >= mt && t <= 1.0f - mt) inter = 1;
            else if (s < -ms || s > 1.0f + ms || t < -mt || t > 1.0f + mt) inter = 0;
        }
    }
    float tt;
    const float de[4] = {seg_param(P0, Q0, Q1, tt), seg_param(P1, Q0, Q1, tt), seg_param(Q0, P0, P1, tt),
                         seg_param(Q1, P0, P1, tt)};
    float emin = fminf(fminf(de[0], de[1]), fminf(de[2], de[3]));
    if (best > 2.9e38f || emin < best) best = emin;
    dmin = sqrtf(best);
    if (inter == 1) return 1;
    const float r = sqrtf(emin), lim = r + 2.0f * cert_err(ex, r), lim2 = lim * lim;
    int mask = inter < 0 ? 1 : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (de[j] <= lim2) mask |= 2 << j;
    return mask;
}

// r of a feature for slot positions X[4]
template <typename T>
__device__ __forceinline__ V3<T> feat_r(const Feature<T>& f, const V3<T> X[4]) {
    V3<T> r = {T(0), T(0), T(0)};
#pragma unroll
    for (int s = 0; s < 4; ++s) r = r + f.w[s] * X[s];
    return r;
}

// First and second derivative of d along slot directions dl[4] (sensitivity
// of the closest-point problem restricted to the active feature):
//   D = d^2, D' = 2 r.rdot, D'' = 2|rdot|^2 - 2 b^T (J^T J)^-1 b,
//   J_k = sum_s e_ks X_s, b_k = (sum_s e_ks dl_s).r + J_k.rdot,
//   d' = D'/(2d), d'' = (D'' - 2 d'^2) / (2d).
template <typename T>
__device__ __forceinline__ void feat_dir_derivs(const Feature<T>& f, const V3<T> X[4], const V3<T> dl[4], T& d1,
                                                T& d2) {
    V3<T> r = feat_r(f, X);
    V3<T> rd = {T(0), T(0), T(0)};
#pragma unroll
    for (int s = 0; s < 4; ++s) rd = rd + f.w[s] * dl[s];
    T D2 = T(2) * dot(rd, rd);
    if (f.nf > 0) {
        V3<T> J[2], Gk[2];
        T bk[2];
        for (int k = 0; k < f.nf; ++k) {
            J[k] = {T(0), T(0), T(0)};
            Gk[k] = {T(0), T(0), T(0)};
            for (int s = 0; s < 4; ++s) {
                J[k] = J[k] + f.e[k][s] * X[s];
                Gk[k] = Gk[k] + f.e[k][s] * dl[s];
            }
            bk[k] = dot(Gk[k], r) + dot(J[k], rd);
        }
        if (f.nf == 1) {
            T m = dot(J[0], J[0]);
            if (m > T(0)) D2 -= T(2) * bk[0] * bk[0] / m;
        } else {
            T m00 = dot(J[0], J[0]), m01 = dot(J[0], J[1]), m11 = dot(J[1], J[1]);
            T det = m00 * m11 - m01 * m01;
            if (det > T(0)) D2 -= T(2) * (m11 * bk[0] * bk[0] - T(2) * m01 * bk[0] * bk[1] + m00 * bk[1] * bk[1]) / det;
        }
    }
    d1 = dot(r, rd) / f.d;
    d2 = (D2 - T(2) * d1 * d1) / (T(2) * f.d);
}

// Action of the distance Hessian on slot directions dl (same sensitivity):
// the optimal free parameters move by thd = -(J^T J)^-1 b, the closest-point
// vector by rt = rdot + sum_k thd_k J_k, and per slot
//   (grad^2 d . dl)_s = (sum_k thd_k e_ks) rhat + w_s (I - rhat rhat^T) rt / d.
// Also returns d1 = rhat . rdot and rhat.
__device__ __forceinline__ void feat_hess_vec(const Feature<double>& f, const V3<double> X[4], const V3<double> dl[4],
                                              double& d1, V3<double> hv[4], V3<double>& rh) {
    V3<double> r = feat_r(f, X);
    rh = (1.0 / f.d) * r;
    V3<double> rd = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < 4; ++s) rd = rd + f.w[s] * dl[s];
    double thd[2] = {0.0, 0.0};
    V3<double> J[2] = {{0, 0, 0}, {0, 0, 0}};
    if (f.nf > 0) {
        V3<double> Gk[2];
        double bk[2];
        for (int k = 0; k < f.nf; ++k) {
            Gk[k] = {0, 0, 0};
            for (int s = 0; s < 4; ++s) {
                J[k] = J[k] + f.e[k][s] * X[s];
                Gk[k] = Gk[k] + f.e[k][s] * dl[s];
            }
            bk[k] = dot(Gk[k], r) + dot(J[k], rd);
        }
        if (f.nf == 1) {
            double m = dot(J[0], J[0]);
            if (m > 0) thd[0] = -bk[0] / m;
        } else {
            double m00 = dot(J[0], J[0]), m01 = dot(J[0], J[1]), m11 = dot(J[1], J[1]);
            double det = m00 * m11 - m01 * m01;
            if (det > 0) {
                thd[0] = -(m11 * bk[0] - m01 * bk[1]) / det;
                thd[1] = -(m00 * bk[1] - m01 * bk[0]) / det;
            }
        }
    }
    V3<double> rt = rd + thd[0] * J[0] + thd[1] * J[1];
    V3<double> tang = rt - dot(rh, rt) * rh;
    double inv = 1.0 / f.d;
#pragma unroll
    for (int s = 0; s < 4; ++s) hv[s] = (thd[0] * f.e[0][s] + thd[1] * f.e[1][s]) * rh + (f.w[s] * inv) * tang;
    d1 = dot(rh, rd);
}

// ---------------------------------------------------------------------------
// Parallel-edge mollifier of the edge-edge terms (IPC, Li et al. 2020): an
// edge-edge pair contributes m(c) b(d) with c = |u x v|^2, u = X1 - X0 and
// v = X3 - X2 over its slots [P0, P1, Q0, Q1], and
//   m(c) = (2 - c/eps) c/eps for c < eps, else 1,
// eps = 1e-3 |rest u|^2 |rest v|^2. The edge-edge distance has a kink where
// the edges turn parallel, the configuration a pressed edge settles into;
// m makes the term C^1 there. eps = 0 (point-triangle pairs) gives m = 1.

template <typename T>
struct EdgeMollT {
    T m, m1, m2;              // m(c), m'(c), m''(c)
    V3<T> u, v, w;            // the two edges and w = u x v
    bool on;                  // c < eps: the derivatives of m enter
};
using EdgeMoll = EdgeMollT<double>;

template <typename T>
__device__ __forceinline__ EdgeMollT<T> edge_moll(const V3<T> X[4], T eps) {
    EdgeMollT<T> e;
    e.u = X[1] - X[0];
    e.v = X[3] - X[2];
    e.w = cross(e.u, e.v);
    const T c = dot(e.w, e.w);
    e.on = eps > T(0) && c < eps;
    if (e.on) {
        const T ie = T(1) / eps, q = c * ie;
        e.m = (T(2) - q) * q;
        e.m1 = T(2) * ie * (T(1) - q);
        e.m2 = T(-2) * ie * ie;
    } else {
        e.m = T(1);
        e.m1 = T(0);
        e.m2 = T(0);
    }
    return e;
}

// dc/dX of slot s: dc = 2 (v x w).du + 2 (w x u).dv
template <typename T>
__device__ __forceinline__ V3<T> edge_moll_grad(const EdgeMollT<T>& e, int s) {
    V3<T> g = s < 2 ? cross(e.v, e.w) : cross(e.w, e.u);
    const T sg = (s == 0 || s == 2) ? T(-2) : T(2);
    return sg * g;
}

// c' and c'' along slot directions dl: with s = du x v + u x dv,
// c' = 2 w.s and c'' = 2 |s|^2 + 4 w.(du x dv)
template <typename T>
__device__ __forceinline__ void edge_moll_dir(const EdgeMollT<T>& e, const V3<T> dl[4], T& c1, T& c2) {
    const V3<T> du = dl[1] - dl[0], dv = dl[3] - dl[2];
    const V3<T> s = cross(du, e.v) + cross(e.u, dv);
    c1 = T(2) * dot(e.w, s);
    c2 = T(2) * dot(s, s) + T(4) * dot(e.w, cross(du, dv));
}

// (Hess c) dl of slot s: the gradient of c' = 2 w.s for fixed dl,
// d/du = 2 (v x s) + 2 (dv x w), d/dv = 2 (s x u) + 2 (w x du)
__device__ __forceinline__ V3<double> edge_moll_hvec(const EdgeMoll& e, const V3<double> dl[4], int s) {
    const V3<double> du = dl[1] - dl[0], dv = dl[3] - dl[2];
    const V3<double> sv = cross(du, e.v) + cross(e.u, dv);
    V3<double> h = s < 2 ? cross(e.v, sv) + cross(dv, e.w) : cross(sv, e.u) + cross(e.w, du);
    const double sg = (s == 0 || s == 2) ? -2.0 : 2.0;
    return sg * h;
}

// Second derivative of m(c) b(d) along slot directions, from d', d'' (the
// feature's directional derivatives) and b, b', b'' at d:
//   m (b'' d'^2 + b' d'') + m'' c'^2 b + m' c'' b + 2 m' c' b' d'
template <typename T>
__device__ __forceinline__ T moll_barrier_dir2(const EdgeMollT<T>& e, const V3<T> dl[4], T d1, T d2,
                                               const Barrier3T<T>& bb) {
    T q = bb.b2 * d1 * d1 + bb.b1 * d2;
    if (!e.on) return q;
    T c1, c2;
    edge_moll_dir(e, dl, c1, c2);
    return e.m * q + e.m2 * c1 * c1 * bb.b + e.m1 * c2 * bb.b + T(2) * e.m1 * c1 * bb.b1 * d1;
}

// ---------------------------------------------------------------------------
// Friction mollifier f(s) of Eq. (friction_mollifier) and helpers.

template <typename T>
__device__ __forceinline__ T moll_f(T s, T eps) {
    return s < eps ? -s * s * s / (T(3) * eps * eps) + s * s / eps + eps / T(3) : s;
}
template <typename T>
__device__ __forceinline__ T moll_f1_over_s(T s, T eps) {
    return s < eps ? -s / (eps * eps) + T(2) / eps : T(1) / s;
}
// coefficient c(s) of the u u^T term of the tangent Hessian
template <typename T>
__device__ __forceinline__ T moll_c(T s, T eps) {
    return s < eps ? s / (eps * eps) : (s > T(0) ? T(1) / s : T(0));
}

// ---------------------------------------------------------------------------
// 3x3 symmetric block helpers; blocks are stored (xx, yy, zz, xy, xz, yz).

__device__ __forceinline__ bool sym_inverse(const float K[6], float Kinv[6]) {
    float a = K[0], b = K[1], c = K[2], d = K[3], e = K[4], f = K[5];
    float c00 = b * c - f * f, c01 = e * f - d * c, c02 = d * f - b * e;
    float det = a * c00 + d * c01 + e * c02;
    if (!(det > 0.0f)) return false;
    float id = 1.0f / det;
    Kinv[0] = c00 * id;
    Kinv[1] = (a * c - e * e) * id;
    Kinv[2] = (a * b - d * d) * id;
    Kinv[3] = c01 * id;
    Kinv[4] = c02 * id;
    Kinv[5] = (d * e - a * f) * id;
    return true;
}

__device__ __forceinline__ void sym_apply(const float K[6], const float v[3], float o[3]) {
    o[0] = K[0] * v[0] + K[3] * v[1] + K[4] * v[2];
    o[1] = K[3] * v[0] + K[1] * v[1] + K[5] * v[2];
    o[2] = K[4] * v[0] + K[5] * v[1] + K[2] * v[2];
}

}  // namespace tac
