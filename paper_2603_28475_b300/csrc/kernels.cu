// Kernels of the PNCG-IPC gel-pad solve (see solve.cuh for the data layout).
//
// Readings of the paper that these kernels share with the FP64 oracle:
//  * step alpha = min(dhat / (2 max_i |p_i|), alpha_ccd, -g^T p / p^T H p)
//    (Eq. step_size plus a conservative per-pair bound eta d_k / max |p_i|),
//    then Armijo backtracking on E(x + alpha p) - E(x) <= c alpha g^T p,
//    evaluated as alpha g(x + alpha p)^T p - R'(alpha) with R' the
//    element-wise second-order remainder expanded at the trial point;
//    the pad's step mode 1 is Eq. (step_size) as printed: alpha =
//    min(alpha_upper, alpha_bar), no CCD bound and no energy test (a trial
//    state outside E's domain is still halved);
//  * beta of Eq. (dk_direction); restart when y^T p is negligible or the new
//    direction is not a descent direction;
//  * the indenter moves on the straight per-vertex path between its frame
//    poses in substeps of eta * d_min / max |y^{t+1} - y^t|;
//  * the candidate set is rebuilt before the accumulated motion bound since
//    the last build exceeds the margin m = dhat.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "solve.cuh"

// TAC_WIDE (kernels_wide.cu) compiles the persistent solve kernel a second
// time in the 512-thread block shape, in namespace tac::wide; everything
// else of this file is compiled once, in the 256-thread shape.
#ifdef TAC_WIDE
namespace tac {
namespace wide {
constexpr int kThreads = 512;         // 16 warps, one CTA per SM
constexpr int kCtasPerSm = 1;
#else
namespace tac {
constexpr int kCtasPerSm = 2;
#endif

constexpr float kEta = 0.9f;          // safety factor of the step bounds
constexpr double kArmijoC = 1e-4;
constexpr int kMaxHalvings = 20;
constexpr int kMaxSubsteps = 4000;
constexpr int kWarps = kThreads / 32;
// the host balances the colour classes for rounds of kCtaWarps patches; a
// wider CTA runs the same classes in rounds of its own warp count
static_assert(kWarps % kCtaWarps == 0, "a CTA runs whole rounds of the host's colour classes");
// A pair whose float32 distance exceeds kNearBand * dhat is outside the
// barrier's support in float64 as well: at the workloads' coordinate
// magnitudes (a few cm) the float32 distance is off by ~1e-8 m at most,
// far below the band's 0.05 dhat. Such pairs skip the float64 feature.
constexpr double kNearBand = 1.05;

// ---------------------------------------------------------------------------
// shared memory of one CTA

// raw data of one warp-sized tet patch, copied asynchronously from global
// memory (one tet and one vertex per lane)
struct PatchStage {
    float B[9][32];             // Dm^-1 entries of the patch's tets
    uint32_t lc[32];            // 4 x 8-bit local vertex ids (kNoTet: unused slot)
    uint32_t sl[32];            // 4 x 8-bit corner slots
    float uh[3][32];            // displacement (hi) of the patch's vertices
    float ul[3][32];            // displacement (lo)
    float p[3][32];             // direction
    float og[9][32];            // scatter passes: the vertices' sums so far (gradient, blocks)
};

// Corner slot s of a patch lives at s + s / 32 in the corner stage: a
// vertex's run starts near 4 x its local id, so without the padding word per
// 32 slots the lanes 8 apart would read the same bank in the scatter.
constexpr int kStagePad = kStage + kStage / 32;
__device__ __forceinline__ int stg_pos(int s) { return s + (s >> 5); }

// per-warp scratch of the tet passes
struct WarpScratch {
    PatchStage st[2];           // double buffer: the warp's next patch loads while this one computes
    float stg[6][kStagePad];    // corner values of the current patch: force (3) and, in the gradient
                                // pass, s = sqrt(hV coef) c whose outer product is the block's
                                // non-static part
};

struct Shared {
    WarpScratch w[kWarps];
    PadDev P;                   // descriptors of the CTA's current pad (see load_pad)
    MeshDev M;
    EnvDev E;
    double rd[kWarps][8];
    double rsum[8];
    float rf[kWarps][4];
    int ri[kWarps];
    int cnt[4];
    float box[12];
    int pad;
    int flag;
    int fok;                    // D.fcache holds the float64 features of the current point and pair set
    float dm[kMaxDmTypes * 9];  // the current pad's Dm^-1 table (meshes with n_dm > 0)
};

// one CTA-wide scratch object (dynamic shared memory, sizeof(Shared) bytes at
// every launch), visible to every device function of the file
extern __shared__ __align__(16) unsigned char tac_smem[];
#define S (*reinterpret_cast<Shared*>(tac_smem))

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// per-phase wall time of one pad's solve, accumulated by thread 0 at points
// where the CTA is already synchronised
enum { PH_TET0 = 0, PH_TET1, PH_PAIR_PHP, PH_PAIR_TRIAL, PH_VERTEX, PH_BROAD, PH_SETUP, PH_COUNT };

struct PhaseClock {
    unsigned long long last = 0;
    unsigned long long acc[PH_COUNT] = {0, 0, 0, 0, 0, 0, 0};
    __device__ __forceinline__ void start() {
        if (threadIdx.x == 0) last = global_ns();
    }
    __device__ __forceinline__ void lap(int ph) {
        if (threadIdx.x == 0) {
            unsigned long long t = global_ns();
            acc[ph] += t - last;
            last = t;
        }
    }
};

// The CTA's pad descriptors, identical for all its threads, go to shared
// memory once per pad: the phase functions take them by reference, and a
// per-thread copy would live on the stack and be re-read from local memory.
__device__ __forceinline__ void load_pad(const Dev& D, int pad) {
    if (threadIdx.x == 0) {
        S.P = D.pads[pad];
        S.M = D.meshes[S.P.mesh];
        S.E = D.envs[S.P.env];
        S.fok = 0;
    }
    __syncthreads();
    const int ndm = S.M.n_dm;
    if (ndm > 0) {
        for (int i = threadIdx.x; i < 9 * ndm; i += blockDim.x) S.dm[i] = D.dm_table[9 * S.M.dm_off + i];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// block-wide helpers (every thread receives the same result)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// K <= 8 sums; thread k adds the warps' partial sums of value k in warp
// order, so every thread receives the same, order-fixed result
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
    static_assert(K <= 8, "block_sum holds at most 8 values");
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) S.rd[w][k] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < kWarps; ++i) t += S.rd[i][threadIdx.x];
        S.rsum[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = S.rsum[k];
}

// K <= 4 float sums in float arithmetic (the plain-FP32 form's reductions),
// order-fixed like block_sum
template <int K>
__device__ __forceinline__ void block_sum_f32(float (&v)[K]) {
    static_assert(K <= 4, "block_sum_f32 holds at most 4 values");
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) S.rf[w][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < kWarps; ++i) t += S.rf[i][k];
        v[k] = t;
    }
    __syncthreads();
}

// Block sum of K per-thread values of type R: float64 for the chosen form,
// float for the plain-FP32 form
template <typename R, int K>
__device__ __forceinline__ void block_sum_r(R (&v)[K]) {
    if constexpr (sizeof(R) == 8) {
        block_sum<K>(v);
    } else {
        block_sum_f32<K>(v);
    }
}

// Running sum of float terms without float64 arithmetic (FP64 is a narrow
// pipe on this part): hi is the float sum, lo collects the exact rounding
// error of each addition (Knuth's TwoSum), so hi + lo carries the sum to
// about 2^-44 relative. Each term enters as the float it is computed as.
struct FSum {
    float hi, lo;
};

__device__ __forceinline__ void fsum_add(FSum& a, float b) {
    float s = __fadd_rn(a.hi, b);
    float bp = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ double fsum_value(const FSum& a) { return (double)a.hi + (double)a.lo; }

// plain float accumulation (the plain-FP32 form) or TwoSum pairs
__device__ __forceinline__ void fsum_add_mode(FSum& a, float b, bool plain) {
    if (plain)
        a.hi = __fadd_rn(a.hi, b);
    else
        fsum_add(a, b);
}

// Block sums of K running sums: float64 of each thread's (hi + lo) for the
// chosen form, float of each thread's hi for the plain-FP32 form
template <int K>
__device__ __forceinline__ void block_sum_fsum(const FSum (&a)[K], double (&out)[K], bool plain) {
    if (plain) {
        float f[K];
#pragma unroll
        for (int k = 0; k < K; ++k) f[k] = a[k].hi;
        block_sum_f32<K>(f);
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = (double)f[k];
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = fsum_value(a[k]);
        block_sum<K>(out);
    }
}

__device__ __forceinline__ double block_min_d(double v) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) S.rd[w][7] = v;
    __syncthreads();
    double t = S.rd[0][7];
#pragma unroll
    for (int i = 1; i < kWarps; ++i) t = fmin(t, S.rd[i][7]);
    __syncthreads();
    return t;
}

// max of up to 4 floats
template <int K>
__device__ __forceinline__ void block_max_f(float (&v)[K]) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) S.rf[w][k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float t = S.rf[0][k];
#pragma unroll
        for (int i = 1; i < kWarps; ++i) t = fmaxf(t, S.rf[i][k]);
        v[k] = t;
    }
    __syncthreads();
}

// exclusive scan of one int per thread; total to every thread
__device__ __forceinline__ int block_scan(int v, int& total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) S.ri[w] = x;
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) {
        int c = S.ri[i];
        before += (i < w) ? c : 0;
        tot += c;
    }
    __syncthreads();
    total = tot;
    return before + x - v;
}

// ---------------------------------------------------------------------------
// positions

struct Ctx {
    const Dev& D;
    const PadDev& P;
    const MeshDev& M;
    const EnvDev& E;
};

__device__ __forceinline__ double gel_pos64(const Dev& D, const PadDev& P, const MeshDev& M, int gv, int c,
                                            float alpha) {
    int si = c * D.Vt + P.v_off + gv;
    return (double)D.X[c * D.XVt + M.xv_off + gv] + (double)D.uh[si] + (double)D.ul[si] +
           (double)(alpha * D.p[si]);
}

__device__ __forceinline__ float gel_pos32(const Dev& D, const PadDev& P, const MeshDev& M, int gv, int c,
                                           float alpha) {
    int si = c * D.Vt + P.v_off + gv;
    return D.X[c * D.XVt + M.xv_off + gv] + ((D.uh[si] + D.ul[si]) + alpha * D.p[si]);
}

// indenter vertex j (env-local) of this pad at path parameter s
__device__ __forceinline__ double ind_pos64(const Dev& D, const PadDev& P, int j, int c, double s) {
    double a = D.Yt[3 * (P.yw_off + j) + c], b = D.Yn[3 * (P.yw_off + j) + c];
    return a + s * (b - a);
}
__device__ __forceinline__ float ind_pos32(const Dev& D, const PadDev& P, int j, int c, float s) {
    float a = D.Yt[3 * (P.yw_off + j) + c], b = D.Yn[3 * (P.yw_off + j) + c];
    return a + s * (b - a);
}

// slots of a candidate pair: gel mesh vertex ids (or -1) and indenter env
// vertex ids (or -1), canonical order [gel..., indenter...]
__device__ __forceinline__ void pair_slots(const Dev& D, const MeshDev& M, const EnvDev& E, int4 q, int gsl[4],
                                           int isl[4]) {
#pragma unroll
    for (int s = 0; s < 4; ++s) gsl[s] = isl[s] = -1;
    if (q.x == 0) {
        gsl[0] = q.y;
        const int* t = D.it + 3 * (E.t_off + q.z);
        isl[1] = t[0]; isl[2] = t[1]; isl[3] = t[2];
    } else if (q.x == 1) {
        const int* t = D.st + 3 * (M.st_off + q.y);
        gsl[0] = t[0]; gsl[1] = t[1]; gsl[2] = t[2];
        isl[3] = q.z;
    } else {
        const int* e = D.se + 2 * (M.se_off + q.y);
        gsl[0] = e[0]; gsl[1] = e[1];
        const int* f = D.ie + 2 * (E.e_off + q.z);
        isl[2] = f[0]; isl[3] = f[1];
    }
}

// mollifier threshold of a pair: 1e-3 |rest gel edge|^2 |indenter edge|^2
// for an edge-edge pair (slots [gel a, gel b, indenter a, indenter b]), 0
// for the point-triangle types
__device__ __forceinline__ double ee_eps(const Dev& D, const MeshDev& M, const EnvDev& E, int type, const int gsl[4],
                                         const int isl[4]) {
    if (type != 2) return 0.0;
    double a2 = 0.0, b2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double a = (double)D.X[c * D.XVt + M.xv_off + gsl[1]] - (double)D.X[c * D.XVt + M.xv_off + gsl[0]];
        const double b = (double)D.Y[3 * (E.y_off + isl[3]) + c] - (double)D.Y[3 * (E.y_off + isl[2]) + c];
        a2 += a * a;
        b2 += b * b;
    }
    return 1e-3 * a2 * b2;
}

// feature of a pair from slot positions; type 1 is re-expressed with the gel
// triangle first and r pointing from the indenter to the gel
// (mask: the candidates to search, from pair_pick; all by default)
template <typename T>
__device__ __forceinline__ Feature<T> pair_feature(int type, const V3<T> X[4], int mask = 31) {
    if (type == 0) return pt_feature<T>(X[0], X[1], X[2], X[3], mask & 15);
    if (type == 2) return ee_feature<T>(X[0], X[1], X[2], X[3], mask);
    Feature<T> f = pt_feature<T>(X[3], X[0], X[1], X[2], mask & 15);
    Feature<T> g;
    g.d = f.d;
    g.nf = f.nf;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        g.w[s] = -f.w[s + 1];
        g.e[0][s] = -f.e[0][s + 1];
        g.e[1][s] = -f.e[1][s + 1];
    }
    g.w[3] = -f.w[0];
    g.e[0][3] = -f.e[0][0];
    g.e[1][3] = -f.e[1][0];
    return g;
}

template <typename T>
__device__ __forceinline__ void load_slots(const Dev& D, const PadDev& P, const MeshDev& M, const int gsl[4],
                                           const int isl[4], float alpha, double s, V3<T> X[4]);

template <>
__device__ __forceinline__ void load_slots<double>(const Dev& D, const PadDev& P, const MeshDev& M,
                                                   const int gsl[4], const int isl[4], float alpha, double s,
                                                   V3<double> X[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (gsl[k] >= 0)
            X[k] = {gel_pos64(D, P, M, gsl[k], 0, alpha), gel_pos64(D, P, M, gsl[k], 1, alpha),
                    gel_pos64(D, P, M, gsl[k], 2, alpha)};
        else
            X[k] = {ind_pos64(D, P, isl[k], 0, s), ind_pos64(D, P, isl[k], 1, s), ind_pos64(D, P, isl[k], 2, s)};
    }
}

template <>
__device__ __forceinline__ void load_slots<float>(const Dev& D, const PadDev& P, const MeshDev& M,
                                                  const int gsl[4], const int isl[4], float alpha, double s,
                                                  V3<float> X[4]) {
    float sf = (float)s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (gsl[k] >= 0)
            X[k] = {gel_pos32(D, P, M, gsl[k], 0, alpha), gel_pos32(D, P, M, gsl[k], 1, alpha),
                    gel_pos32(D, P, M, gsl[k], 2, alpha)};
        else
            X[k] = {ind_pos32(D, P, isl[k], 0, sf), ind_pos32(D, P, isl[k], 1, sf), ind_pos32(D, P, isl[k], 2, sf)};
    }
}

// Float32 distance of a pair and the mask of the closest-feature candidates
// that can win its float64 search (pt_mask / ee_mask on the slots in
// pair_feature's order). The float32 slot positions are within 2 units of
// 2^-24 of the largest coordinate of the float64 ones (one rounding of the
// sum and one of the interpolated indenter vertex); ex takes 8.
__device__ __forceinline__ float pair_pick(int type, const V3<float> X[4], int& mask) {
    float xm = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s) xm = fmaxf(xm, fmaxf(fabsf(X[s].x), fmaxf(fabsf(X[s].y), fabsf(X[s].z))));
    const float ex = 4.76837158203125e-7f * xm;
    float d;
    if (type == 0) mask = pt_mask(X[0], X[1], X[2], X[3], ex, d);
    else if (type == 2) mask = ee_mask(X[0], X[1], X[2], X[3], ex, d);
    else mask = pt_mask(X[3], X[0], X[1], X[2], ex, d);
    return d;
}

// distance of a pair: float32 estimate, float64 when close (relative band);
// the plain-FP32 form takes the float32 distance
template <typename R>
__device__ __forceinline__ R pair_distance(const Dev& D, const PadDev& P, const MeshDev& M, int type,
                                           const int gsl[4], const int isl[4], float alpha, double s, double near) {
    V3<float> Xf[4];
    load_slots<float>(D, P, M, gsl, isl, alpha, s, Xf);
    if constexpr (sizeof(R) == 4) {
        return pair_feature<float>(type, Xf).d;   // the plain-FP32 form
    } else {
        int mask;
        const float df = pair_pick(type, Xf, mask);
        if ((double)df > near) return (double)df * (1.0 - 1e-5);
        V3<double> Xd[4];
        load_slots<double>(D, P, M, gsl, isl, alpha, s, Xd);
        return pair_feature<double>(type, Xd, mask).d;
    }
}

// ---------------------------------------------------------------------------
// tet passes

struct TetOut {
    double acc;       // p^T H_e p (pass 0), remainder R' (pass 1), lambda-sensitivity (pass 3)
    int bad;          // trial state inverted a tet
    float fmax;       // largest per-corner force component (pass 1)
    double acc2;      // mu-sensitivity (pass 3)
};

// The tet passes read their arrays through these pointers, taken from the
// batch and pad descriptors once per pass: the descriptors are reached through
// references, and their fields would otherwise be reloaded after every store.
struct TetPtrs {
    const float* B;             // Dm^-1 of the pad's mesh (stride Tt between entries)
    const uint32_t* lc;         // local vertex ids
    const uint32_t* sl;         // corner slots
    const float* uh;            // state of the pad (stride Vt between components)
    const float* ul;
    const float* p;
    float* g;
    float* blk;
    const float* wd;            // static block diagonal of the mesh's vertices
    const int* pv;              // patch vertex entries
    const uint16_t* pc;         // patch CSR offsets
    size_t Tt, Vt;
};

__device__ __forceinline__ TetPtrs tet_ptrs(const Dev& D, const PadDev& P, const MeshDev& M, int gb) {
    TetPtrs T;
    T.B = D.B + M.tet_off;
    T.lc = D.lconn + M.tet_off;
    T.sl = D.slot + M.tet_off;
    T.uh = D.uh + P.v_off;
    T.ul = D.ul + P.v_off;
    T.p = D.p + P.v_off;
    T.g = D.g[gb] + P.v_off;
    T.blk = D.blk[gb] + P.v_off;
    T.wd = D.wdiag + M.xv_off;
    T.pv = D.pvert + M.pvert_off;
    T.pc = D.pcsr + M.pcsr_off;
    T.Tt = D.Tt;
    T.Vt = D.Vt;
    return T;
}

// asynchronous copy of one warp patch into a stage; lane k copies tet slot k
// and, when the patch has a vertex entry k (gvf >= 0), that vertex's data.
// The scatter passes also copy the vertex's sums so far when this is not its
// first patch: patches of one colour class share no vertex and earlier
// classes are complete, so those sums are final when the copy is issued.
template <int PASS, bool TAB>
__device__ __forceinline__ void issue_patch(const TetPtrs& T, int pi, int gvf, PatchStage& st, int lane) {
    {
        size_t t = (size_t)kPatchTets * pi + lane;
        if (!TAB) {
#pragma unroll
            for (int e = 0; e < 9; ++e) cp_async4(&st.B[e][lane], T.B + (size_t)e * T.Tt + t);
        }
        cp_async4(&st.lc[lane], T.lc + t);
        cp_async4(&st.sl[lane], T.sl + t);
    }
    if (gvf >= 0) {
        const int lv = gvf & kVertMask;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cp_async4(&st.uh[c][lane], T.uh + (size_t)c * T.Vt + lv);
            cp_async4(&st.ul[c][lane], T.ul + (size_t)c * T.Vt + lv);
            cp_async4(&st.p[c][lane], T.p + (size_t)c * T.Vt + lv);
        }
        if ((PASS == 1 || PASS == 2) && !(gvf & kFirstFlag)) {
#pragma unroll
            for (int c = 0; c < 3; ++c) cp_async4(&st.og[c][lane], T.g + (size_t)c * T.Vt + lv);
            if (PASS == 1) {
#pragma unroll
                for (int c = 0; c < 6; ++c) cp_async4(&st.og[3 + c][lane], T.blk + (size_t)c * T.Vt + lv);
            }
        } else if (PASS == 1) {
            // first patch of the vertex: the blocks' static diagonal enters here
            cp_async4(&st.og[3][lane], T.wd + lv);
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ int patch_vert(const TetPtrs& T, int pi, int lane) {
    return __ldg(T.pv + kPatchVerts * pi + lane);
}

// pass 0: p^T H_e p at u; pass 1: gradient, diagonal blocks and remainder at
// u + alpha p into g[gb], blk[gb]; pass 2: H_e p into g[gb]; pass 3: lambda
// (in p) against the Lame derivatives of the stress.
// Each warp streams its own patches (one tet per lane) through a private
// double-buffered stage and sums its patch's corner contributions per vertex
// (one vertex per lane) before writing them: no CTA barrier inside a colour
// class. Passes that scatter walk the colour classes in order with one CTA
// barrier between classes (patches of one class share no vertex); the
// reduction passes walk all patches without any.
template <int PASS, bool TAB>
__device__ __noinline__ TetOut tet_pass_impl(const Dev& D, const PadDev& P, const MeshDev& M, float alpha, int gb) {
    TetOut out{0.0, 0, 0.f, 0.0};
    FSum acc{0.f, 0.f}, acc2{0.f, 0.f};
    const bool plain = P.prec != 0 && PASS < 2;   // plain-FP32 form: float sums
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    WarpScratch& W = S.w[warp];
    const float mu = P.mu, lam = P.lam, h2 = P.h * P.h;
    const TetPtrs T = tet_ptrs(D, P, M, gb);
    const int* colour = D.colour + M.col_off;
    const int n_patch = M.n_patch;
    constexpr bool kScatter = (PASS == 1 || PASS == 2);
    const int ncls = kScatter ? M.n_col : 1;
    for (int cls = 0; cls < ncls; ++cls) {
        const int p_begin = kScatter ? __ldg(colour + cls) : 0;
        const int p_end = kScatter ? __ldg(colour + cls + 1) : n_patch;
        int pi = p_begin + warp;
        int b = 0;
        // vertex entries of this lane: current patch (gvf_c), the next one
        // (gvf_n, loaded one patch ahead so that issuing its copy does not wait)
        int gvf_c = -1, gvf_n = -1;
        if (pi < p_end) {
            gvf_c = patch_vert(T, pi, lane);
            issue_patch<PASS, TAB>(T, pi, gvf_c, W.st[0], lane);
            if (pi + kWarps < p_end) gvf_n = patch_vert(T, pi + kWarps, lane);
        }
        while (pi < p_end) {
            const int pn = pi + kWarps;
            cp_async_wait_all();
            __syncwarp();                       // stage b complete for every lane
            int s0 = 0, s1 = 0;
            if (kScatter) {
                s0 = __ldg(T.pc + kPatchCsr * pi + lane);
                s1 = __ldg(T.pc + kPatchCsr * pi + lane + 1);
            }
            int gvf_nn = -1;
            if (pn < p_end) {
                issue_patch<PASS, TAB>(T, pn, gvf_n, W.st[b ^ 1], lane);
                if (pn + kWarps < p_end) gvf_nn = patch_vert(T, pn + kWarps, lane);
            }
            const PatchStage& st = W.st[b];
            const uint32_t lc = st.lc[lane];
            if (lc != kNoTet) {
                int l0 = lc & kLocalMask, l1 = (lc >> 8) & kLocalMask, l2 = (lc >> 16) & kLocalMask,
                    l3 = (lc >> 24) & kLocalMask;
                float Bm[9];
                if (TAB) {
                    const float* bt = S.dm + 9 * dm_type_of(lc);
    #pragma unroll
                    for (int e = 0; e < 9; ++e) Bm[e] = bt[e];
                } else {
    #pragma unroll
                    for (int e = 0; e < 9; ++e) Bm[e] = st.B[e][lane];
                }
                float Du[9], Dp[9];
    #pragma unroll
                for (int r = 0; r < 3; ++r) {
                    float h0 = st.uh[r][l0], o0 = st.ul[r][l0], p0 = st.p[r][l0];
                    float p1 = st.p[r][l1] - p0, p2 = st.p[r][l2] - p0, p3 = st.p[r][l3] - p0;
                    Dp[3 * r + 0] = p1;
                    Dp[3 * r + 1] = p2;
                    Dp[3 * r + 2] = p3;
                    Du[3 * r + 0] = ((st.uh[r][l1] - h0) + (st.ul[r][l1] - o0)) + alpha * p1;
                    Du[3 * r + 1] = ((st.uh[r][l2] - h0) + (st.ul[r][l2] - o0)) + alpha * p2;
                    Du[3 * r + 2] = ((st.uh[r][l3] - h0) + (st.ul[r][l3] - o0)) + alpha * p3;
                }
                float G[9], dF[9];
    #pragma unroll
                for (int r = 0; r < 3; ++r)
    #pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        G[3 * r + c] = Du[3 * r] * Bm[c] + Du[3 * r + 1] * Bm[3 + c] + Du[3 * r + 2] * Bm[6 + c];
                        dF[3 * r + c] = Dp[3 * r] * Bm[c] + Dp[3 * r + 1] * Bm[3 + c] + Dp[3 * r + 2] * Bm[6 + c];
                    }
                float detB = Bm[0] * (Bm[4] * Bm[8] - Bm[5] * Bm[7]) - Bm[1] * (Bm[3] * Bm[8] - Bm[5] * Bm[6]) +
                             Bm[2] * (Bm[3] * Bm[7] - Bm[4] * Bm[6]);
                float hV = h2 / (6.0f * detB);
                FAnalysis f;
                f_analysis(G, f);
                float dF2 = 0.f;
    #pragma unroll
                for (int e = 0; e < 9; ++e) dF2 += dF[e] * dF[e];
                AInv ai = a_invariants(f, dF);
                if (PASS == 0) {
                    fsum_add_mode(acc, hV * (mu * dF2 + (mu - lam * f.lnJ) * ai.trA2 + lam * ai.c1 * ai.c1), plain);
                } else if (PASS == 3) {
                    // direction dF = D_lambda Dm^-1: dP/dlam : dF = ln J tr(F^-1 dF),
                    // dP/dmu : dF = (F - F^-T) : dF = tr dF + G : dF - tr(F^-1 dF)
                    float GdF = 0.f;
    #pragma unroll
                    for (int e = 0; e < 9; ++e) GdF += G[e] * dF[e];
                    fsum_add_mode(acc, hV * f.lnJ * ai.c1, plain);
                    fsum_add_mode(acc2, hV * ((dF[0] + dF[4] + dF[8]) + GdF - ai.c1), plain);
                } else if (PASS == 2) {
                    // dP = mu dF + (mu - lam ln J) F^-T dF^T F^-T + lam tr(F^-1 dF) F^-T
                    float C[9];
    #pragma unroll
                    for (int e = 0; e < 9; ++e) C[e] = f.cof[e] * f.invJ;
                    float M1[9];
    #pragma unroll
                    for (int i = 0; i < 3; ++i)
    #pragma unroll
                        for (int l = 0; l < 3; ++l)
                            M1[3 * i + l] = C[3 * i] * dF[3 * l] + C[3 * i + 1] * dF[3 * l + 1] + C[3 * i + 2] * dF[3 * l + 2];
                    float a2 = mu - lam * f.lnJ, a3 = lam * ai.c1;
                    float dP[9];
    #pragma unroll
                    for (int i = 0; i < 3; ++i)
    #pragma unroll
                        for (int j = 0; j < 3; ++j)
                            dP[3 * i + j] = mu * dF[3 * i + j] +
                                            a2 * (M1[3 * i] * C[j] + M1[3 * i + 1] * C[3 + j] + M1[3 * i + 2] * C[6 + j]) +
                                            a3 * C[3 * i + j];
                    float Hc[3][3];
    #pragma unroll
                    for (int k = 0; k < 3; ++k)
    #pragma unroll
                        for (int r = 0; r < 3; ++r)
                            Hc[k][r] = hV * (dP[3 * r] * Bm[3 * k] + dP[3 * r + 1] * Bm[3 * k + 1] + dP[3 * r + 2] * Bm[3 * k + 2]);
                    uint32_t sl = st.sl[lane];
    #pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        int slot = (int)((sl >> (8 * k)) & 0xff);
    #pragma unroll
                        for (int c = 0; c < 3; ++c)
                            W.stg[c][stg_pos(slot)] = (k == 0) ? -(Hc[0][c] + Hc[1][c] + Hc[2][c]) : Hc[k - 1][c];
                    }
                } else {
                    if (!(f.J > 0.0f)) out.bad = 1;
                    // remainder of the line expanded at the trial point (step -alpha)
                    float q = alpha * (-ai.c1 + alpha * (ai.c2 - alpha * ai.c3));
                    float a2c = alpha * alpha * (ai.c2 - alpha * ai.c3);
                    float dl = log1p_minus(q) + a2c;          // ln det(I - aA) + a tr A
                    float dlnJ = log1pf(q);
                    fsum_add_mode(acc, hV * (0.5f * mu * alpha * alpha * dF2 + (lam * f.lnJ - mu) * dl +
                                              0.5f * lam * dlnJ * dlnJ), plain);
                    // first Piola-Kirchhoff stress P = (mu Q + lam ln J cof) / J
                    float Pm[9];
    #pragma unroll
                    for (int e = 0; e < 9; ++e) Pm[e] = (mu * f.Q[e] + lam * f.lnJ * f.cof[e]) * f.invJ;
                    // H = hV P B^T: column k is the force on corner k+1
                    float Hc[3][3];
    #pragma unroll
                    for (int k = 0; k < 3; ++k)
    #pragma unroll
                        for (int r = 0; r < 3; ++r)
                            Hc[k][r] = hV * (Pm[3 * r] * Bm[3 * k] + Pm[3 * r + 1] * Bm[3 * k + 1] + Pm[3 * r + 2] * Bm[3 * k + 2]);
                    float coef = fmaxf(mu + lam * (1.0f - f.lnJ), 0.0f) * f.invJ * f.invJ;
                    // corner block hV (mu |b|^2 I + coef c c^T): the first term is static
                    // (h^2 mu wdiag per vertex), the second s s^T with s = sqrt(hV coef) c
                    const float sq = sqrtf(hV * coef);
                    uint32_t sl = st.sl[lane];
    #pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float bv[3], fo[3];
                        if (k == 0) {
    #pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                bv[c] = -(Bm[c] + Bm[3 + c] + Bm[6 + c]);
                                fo[c] = -(Hc[0][c] + Hc[1][c] + Hc[2][c]);
                            }
                        } else {
    #pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                bv[c] = Bm[3 * (k - 1) + c];
                                fo[c] = Hc[k - 1][c];
                            }
                        }
                        float cc[3];
    #pragma unroll
                        for (int r = 0; r < 3; ++r) cc[r] = f.cof[3 * r] * bv[0] + f.cof[3 * r + 1] * bv[1] + f.cof[3 * r + 2] * bv[2];
                        int slot = stg_pos((int)((sl >> (8 * k)) & 0xff));
                        out.fmax = fmaxf(out.fmax, fmaxf(fabsf(fo[0]), fmaxf(fabsf(fo[1]), fabsf(fo[2]))));
                        W.stg[0][slot] = fo[0];
                        W.stg[1][slot] = fo[1];
                        W.stg[2][slot] = fo[2];
                        W.stg[3][slot] = sq * cc[0];
                        W.stg[4][slot] = sq * cc[1];
                        W.stg[5][slot] = sq * cc[2];
                    }
                }
            }

            if (PASS == 2) {
                __syncwarp();                   // every corner of the patch staged
                if (gvf_c >= 0) {
                    int gv = gvf_c & kVertMask;
                    bool first = (gvf_c & kFirstFlag) != 0;
                    float acc[3] = {0.f, 0.f, 0.f};
                    for (int q = s0; q < s1; ++q)
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[c] += W.stg[c][stg_pos(q)];
#pragma unroll
                    for (int c = 0; c < 3; ++c) T.g[c * T.Vt + gv] = first ? acc[c] : st.og[c][lane] + acc[c];
                }
            }
            if (PASS == 1) {
                __syncwarp();                   // every corner of the patch staged
                if (gvf_c >= 0) {
                    int gv = gvf_c & kVertMask;
                    bool first = (gvf_c & kFirstFlag) != 0;
                    float acc[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) acc[c] = 0.f;
                    for (int q = s0; q < s1; ++q) {
                        const int qp = stg_pos(q);
                        const float f0 = W.stg[0][qp], f1 = W.stg[1][qp], f2 = W.stg[2][qp];
                        const float q0 = W.stg[3][qp], q1 = W.stg[4][qp], q2 = W.stg[5][qp];
                        acc[0] += f0; acc[1] += f1; acc[2] += f2;
                        acc[3] += q0 * q0; acc[4] += q1 * q1; acc[5] += q2 * q2;
                        acc[6] += q0 * q1; acc[7] += q0 * q2; acc[8] += q1 * q2;
                    }
                    if (first) {
                        const float dg = h2 * mu * st.og[3][lane];
#pragma unroll
                        for (int c = 0; c < 3; ++c) T.g[c * T.Vt + gv] = acc[c];
#pragma unroll
                        for (int c = 0; c < 6; ++c) T.blk[c * T.Vt + gv] = c < 3 ? dg + acc[3 + c] : acc[3 + c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; ++c) T.g[c * T.Vt + gv] = st.og[c][lane] + acc[c];
#pragma unroll
                        for (int c = 0; c < 6; ++c) T.blk[c * T.Vt + gv] = st.og[3 + c][lane] + acc[3 + c];
                    }
                }
            }
            __syncwarp();                       // lanes done with stage b and the corner slots
            gvf_c = gvf_n;
            gvf_n = gvf_nn;
            pi = pn;
            b ^= 1;
        }
        if (kScatter) __syncthreads();          // colour class complete: its writes are visible
    }
    // every thread must see the same totals: the caller branches on them
    FSum bad_sum{(float)out.bad, 0.f};
    const FSum sums[3] = {acc, bad_sum, acc2};
    double v[3];
    block_sum_fsum<3>(sums, v, plain);
    out.acc = v[0];
    out.bad = v[1] > 0.0 ? 1 : 0;
    out.acc2 = v[2];
    float fm[1] = {out.fmax};
    block_max_f<1>(fm);
    out.fmax = fm[0];
    return out;
}

// the pass for a mesh with a Dm^-1 table (the tets' rest shapes come from
// shared memory) or with per-tet Dm^-1 (streamed with the patch)
template <int PASS>
__device__ __forceinline__ TetOut tet_pass(const Dev& D, const PadDev& P, const MeshDev& M, float alpha, int gb) {
    return M.n_dm > 0 ? tet_pass_impl<PASS, true>(D, P, M, alpha, gb) : tet_pass_impl<PASS, false>(D, P, M, alpha, gb);
}

// ---------------------------------------------------------------------------
// broad phase: candidate triples (type, i, j) sorted lexicographically

struct BoxF {
    float lo[3], hi[3];
};

// (glo - r) <= ihi and ilo <= (ghi + r) per axis, in float64 on float32
// inputs; a float32 filter decides the cases far from the boundary.
__device__ __forceinline__ bool bp_overlap(const BoxF& g, const BoxF& i, double r, float rlo, float rhi) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float t1 = g.lo[c] - i.hi[c];
        bool a = t1 <= rlo ? true : (t1 > rhi ? false : ((double)g.lo[c] - r) <= (double)i.hi[c]);
        if (!a) return false;
        float t2 = i.lo[c] - g.hi[c];
        bool b = t2 <= rlo ? true : (t2 > rhi ? false : (double)i.lo[c] <= ((double)g.hi[c] + r));
        if (!b) return false;
    }
    return true;
}

__device__ __forceinline__ bool box_near(const BoxF& a, const float* b /*lo3 hi3 inflated*/) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (a.hi[c] < b[c] || a.lo[c] > b[3 + c]) return false;
    return true;
}

// Position sources: the solve state or caller arrays.
struct SrcState {
    const Dev* D;
    const PadDev* P;
    const MeshDev* M;
    float s;
    __device__ float gel(int gv, int c) const { return gel_pos32(*D, *P, *M, gv, c, 0.0f); }
    __device__ float ind(int j, int c) const { return ind_pos32(*D, *P, j, c, s); }
};
// caller positions: gel [n_v][3] in input vertex order (vu: internal ->
// input id, or nullptr when the gel ids are the caller's own), indenter
// [n_ind][3]
struct SrcArrays {
    const float* x;
    const float* y;
    const int* vu;
    __device__ float gel(int gv, int c) const { return x[3 * (vu ? vu[gv] : gv) + c]; }
    __device__ float ind(int j, int c) const { return y[3 * j + c]; }
};

template <class Src>
__device__ __forceinline__ BoxF gel_box(const Src& src, const Dev& D, const MeshDev& M, int type, int i) {
    BoxF b;
    int v[3];
    int n;
    if (type == 0) { v[0] = D.sv[M.sv_off + i]; n = 1; }
    else if (type == 1) { const int* t = D.st + 3 * (M.st_off + i); v[0] = t[0]; v[1] = t[1]; v[2] = t[2]; n = 3; }
    else { const int* e = D.se + 2 * (M.se_off + i); v[0] = e[0]; v[1] = e[1]; n = 2; }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float x = src.gel(v[0], c);
        b.lo[c] = b.hi[c] = x;
        for (int k = 1; k < n; ++k) {
            float y = src.gel(v[k], c);
            b.lo[c] = fminf(b.lo[c], y);
            b.hi[c] = fmaxf(b.hi[c], y);
        }
    }
    return b;
}

template <class Src>
__device__ __forceinline__ BoxF ind_box(const Src& src, const Dev& D, const EnvDev& E, int type, int j) {
    BoxF b;
    int v[3];
    int n;
    if (type == 0) { const int* t = D.it + 3 * (E.t_off + j); v[0] = t[0]; v[1] = t[1]; v[2] = t[2]; n = 3; }
    else if (type == 1) { v[0] = j; n = 1; }
    else { const int* e = D.ie + 2 * (E.e_off + j); v[0] = e[0]; v[1] = e[1]; n = 2; }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float x = src.ind(v[0], c);
        b.lo[c] = b.hi[c] = x;
        for (int k = 1; k < n; ++k) {
            float y = src.ind(v[k], c);
            b.lo[c] = fminf(b.lo[c], y);
            b.hi[c] = fmaxf(b.hi[c], y);
        }
    }
    return b;
}

// Builds the candidate list of one pad into out[0 .. cap); returns the full
// count (> cap means overflow; entries beyond cap are not written).
template <class Src>
__device__ __noinline__ int bp_build(const Src& src, const Dev& D, const MeshDev& M, const EnvDev& E, int* ilist, double r,
                        int4* out, int cap) {
    const int tid = threadIdx.x;
    if (tid == 0) S.fok = 0;             // a new candidate list invalidates cached features
    const float rlo = (float)(r * (1.0 - 1e-5)), rhi = (float)(r * (1.0 + 1e-5));
    const float rc = (float)(r * (1.0 + 1e-4)) + 1e-12f;     // conservative culling radius
    // 1. indenter AABB
    float mx[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX}, mn[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int j = tid; j < E.n_v; j += kThreads)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float y = src.ind(j, c);
            mx[c] = fmaxf(mx[c], y);
            mn[c] = fmaxf(mn[c], -y);
        }
    block_max_f<4>(mx);
    block_max_f<4>(mn);
    float ibox[6] = {-mn[0] - rc, -mn[1] - rc, -mn[2] - rc, mx[0] + rc, mx[1] + rc, mx[2] + rc};
    // 2. union box of gel surface triangles near the indenter box
    float gx[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX}, gn[4] = {-FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int i = tid; i < M.n_st; i += kThreads) {
        BoxF b = gel_box(src, D, M, 1, i);
        if (box_near(b, ibox))
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gx[c] = fmaxf(gx[c], b.hi[c]);
                gn[c] = fmaxf(gn[c], -b.lo[c]);
            }
    }
    block_max_f<4>(gx);
    block_max_f<4>(gn);
    float gbox[6] = {-gn[0] - rc, -gn[1] - rc, -gn[2] - rc, gx[0] + rc, gx[1] + rc, gx[2] + rc};
    bool any_gel = gx[0] > -FLT_MAX;
    // 3. cull indenter primitives of each type against the gel box (order kept)
    int nI[3];
    int base_l[3];
    int nprim[3] = {E.n_t, E.n_v, E.n_e};
    int lbase = 0;
    for (int ty = 0; ty < 3; ++ty) {
        base_l[ty] = lbase;
        int run = 0;
        for (int b0 = 0; b0 < nprim[ty]; b0 += kThreads) {
            int j = b0 + tid;
            int keep = 0;
            if (any_gel && j < nprim[ty]) keep = box_near(ind_box(src, D, E, ty, j), gbox) ? 1 : 0;
            int tot;
            int pos = block_scan(keep, tot);
            if (keep) ilist[lbase + run + pos] = j;
            run += tot;
        }
        nI[ty] = run;
        lbase += nprim[ty];
    }
    // 4. per type: gel primitives in index order, matches in indenter order
    int ngel[3] = {M.n_sv, M.n_st, M.n_se};
    int total = 0;
    for (int ty = 0; ty < 3; ++ty) {
        const int* il = ilist + base_l[ty];
        int nil = nI[ty];
        for (int b0 = 0; b0 < ngel[ty]; b0 += kThreads) {
            int i = b0 + tid;
            int c = 0;
            BoxF gb;
            bool cand = false;
            if (i < ngel[ty] && nil > 0) {
                gb = gel_box(src, D, M, ty, i);
                cand = box_near(gb, ibox);
                if (cand)
                    for (int q = 0; q < nil; ++q) c += bp_overlap(gb, ind_box(src, D, E, ty, il[q]), r, rlo, rhi) ? 1 : 0;
            }
            int tot;
            int pos = block_scan(c, tot) + total;
            if (c > 0) {
                int gi = ty == 0 ? D.sv[M.sv_off + i] : i;
                for (int q = 0; q < nil; ++q) {
                    int j = il[q];
                    if (bp_overlap(gb, ind_box(src, D, E, ty, j), r, rlo, rhi)) {
                        if (pos < cap) out[pos] = make_int4(ty, gi, j, 0);
                        ++pos;
                    }
                }
            }
            total += tot;
        }
    }
    __syncthreads();          // candidate writes visible to the whole CTA
    return total;
}

// ---------------------------------------------------------------------------
// contact entries: per-vertex segmented reduction of pair / lag slot values

struct ContactCtl {
    int npairs, nlag, ncv;
};

__device__ __noinline__ void csr_build(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, ContactCtl& cc) {
    const int tid = threadIdx.x;
    int* cnt = D.cnt + P.v_off;
    int* cvl = D.cvl + 6 * P.pair_off;
    int* cvo = D.cvo + 6 * P.pair_off;
    int* ent = D.ent + 6 * P.pair_off;
    if (tid == 0) S.cnt[0] = 0;
    __syncthreads();
    const int4* pr = D.pairs + P.pair_off;
    const LagRec* lg = D.lag + P.pair_off;
    int np = cc.npairs, nl = cc.nlag;
    for (int k = tid; k < np + nl; k += kThreads) {
        int gs[3];
        if (k < np) {
            int gsl[4], isl[4];
            pair_slots(D, M, E, pr[k], gsl, isl);
            gs[0] = gsl[0]; gs[1] = gsl[1]; gs[2] = gsl[2];
        } else {
            const LagRec& L = lg[k - np];
            gs[0] = L.g[0]; gs[1] = L.g[1]; gs[2] = L.g[2];
        }
        for (int s = 0; s < 3; ++s)
            if (gs[s] >= 0) {
                int old = atomicAdd(&cnt[gs[s]], 1);
                if (old == 0) cvl[atomicAdd(&S.cnt[0], 1)] = gs[s];
            }
    }
    __syncthreads();
    int ncv = S.cnt[0];
    int run = 0;
    for (int b0 = 0; b0 < ncv; b0 += kThreads) {
        int i = b0 + tid;
        int c = i < ncv ? cnt[cvl[i]] : 0;
        int tot;
        int pos = block_scan(c, tot) + run;
        if (i < ncv) cvo[i] = pos;
        run += tot;
    }
    if (tid == 0) cvo[ncv] = run;
    __syncthreads();
    for (int i = tid; i < ncv; i += kThreads) cnt[cvl[i]] = cvo[i];
    __syncthreads();
    for (int k = tid; k < np + nl; k += kThreads) {
        int gs[3];
        if (k < np) {
            int gsl[4], isl[4];
            pair_slots(D, M, E, pr[k], gsl, isl);
            gs[0] = gsl[0]; gs[1] = gsl[1]; gs[2] = gsl[2];
        } else {
            const LagRec& L = lg[k - np];
            gs[0] = L.g[0]; gs[1] = L.g[1]; gs[2] = L.g[2];
        }
        int ebase = k < np ? 3 * k : 3 * (P.pair_cap + (k - np));
        for (int s = 0; s < 3; ++s)
            if (gs[s] >= 0) ent[atomicAdd(&cnt[gs[s]], 1)] = ebase + s;
    }
    __syncthreads();
    for (int i = tid; i < ncv; i += kThreads) {
        int a = cvo[i], b = cvo[i + 1];
        for (int x = a + 1; x < b; ++x) {
            int key = ent[x];
            int y = x - 1;
            while (y >= a && ent[y] > key) {
                ent[y + 1] = ent[y];
                --y;
            }
            ent[y + 1] = key;
        }
        cnt[cvl[i]] = 0;
    }
    __syncthreads();
    cc.ncv = ncv;
}

// adds the slot values of every contact vertex into g[gb], blk[gb]
__device__ __noinline__ void contact_gather(const Dev& D, const PadDev& P, const ContactCtl& cc, int gb) {
    const int* cvl = D.cvl + 6 * P.pair_off;
    const int* cvo = D.cvo + 6 * P.pair_off;
    const int* ent = D.ent + 6 * P.pair_off;
    const float* sb = D.slotbuf + (size_t)9 * 6 * P.pair_off;
    for (int i = threadIdx.x; i < cc.ncv; i += kThreads) {
        float acc[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] = 0.f;
        for (int x = cvo[i]; x < cvo[i + 1]; ++x) {
            const float* e = sb + 9 * ent[x];
#pragma unroll
            for (int c = 0; c < 9; ++c) acc[c] += e[c];
        }
        int si = P.v_off + cvl[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) D.g[gb][c * D.Vt + si] += acc[c];
#pragma unroll
        for (int c = 0; c < 6; ++c) D.blk[gb][c * D.Vt + si] += acc[3 + c];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// pair passes

// minimum distance over the candidates at (u, s)
__device__ __noinline__ double pair_dmin(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np, double s) {
    double dm = 1e300;
    const int4* pr = D.pairs + P.pair_off;
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        dm = fmin(dm, pair_distance<double>(D, P, M, q.x, gsl, isl, 0.0f, s, kNearBand * P.dhat));
    }
    return block_min_d(dm);
}

// p^T H p of the barrier and friction terms and the per-pair step bound at
// the current point; also stores each pair's barrier value b(d) there, which
// the line-search trials of this point subtract from (see pair_trial)
// Float64 features of every pair at the current point u (path parameter s),
// for a pair set that no trial has evaluated yet (a rebuilt candidate list):
// what an accepted trial leaves in the feature cache.
__device__ __noinline__ void pair_cache_fill(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np,
                                             double s) {
    const int4* pr = D.pairs + P.pair_off;
    Feature<double>* fc = D.fcache + P.pair_off;
    const double dh = P.dhat;
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        V3<float> Xf[4];
        load_slots<float>(D, P, M, gsl, isl, 0.0f, s, Xf);
        int mask;
        const float df = pair_pick(q.x, Xf, mask);
        if ((double)df > kNearBand * dh) {
            fc[k].nf = -1;
            fc[k].d = (double)df * (1.0 - 1e-5);
            continue;
        }
        V3<double> X[4];
        load_slots<double>(D, P, M, gsl, isl, 0.0f, s, X);
        fc[k] = pair_feature<double>(q.x, X, mask);
    }
    __syncthreads();
    if (threadIdx.x == 0) S.fok = 1;
    __syncthreads();
}

// p^T H p of the contact and friction terms at u along p, and the CCD bound
// min_k eta d_k / max_slot |p|. The mixed form takes each pair's float64
// feature from what the accepted trial at this point left (pair_cache_fill
// after a rebuild); it stores the barrier values the next trial's remainders
// subtract from.
template <typename R>
__device__ __noinline__ void pair_php(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np, int nl,
                                      double s, double& php, double& accd) {
    constexpr bool kMixed = sizeof(R) == 8;   // float64 features; else the plain-FP32 form
    R acc = R(0), amin = R(3e38);
    const int4* pr = D.pairs + P.pair_off;
    double* bcur = D.bpair + P.pair_off;
    const Feature<double>* fc = D.fcache + P.pair_off;
    if (kMixed && S.fok == 0) pair_cache_fill(D, P, M, E, np, s);
    const R dh = P.dhat, kap = P.kappa;
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        float pk = 0.f;
        V3<float> dl[4];
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            if (gsl[sl] >= 0) {
                int si = P.v_off + gsl[sl];
                float a = D.p[si], b = D.p[D.Vt + si], c = D.p[2 * D.Vt + si];
                pk = fmaxf(pk, sqrtf(a * a + b * b + c * c));
                dl[sl] = {a, b, c};
            } else {
                dl[sl] = {0.f, 0.f, 0.f};
            }
        }
        R d;
        double bv = 0.0;
        if constexpr (kMixed) {
            d = fc[k].d;
            if (fc[k].nf >= 0 && d < dh) {
                V3<double> X[4], dd[4];
                load_slots<double>(D, P, M, gsl, isl, 0.0f, s, X);
#pragma unroll
                for (int sl = 0; sl < 4; ++sl) dd[sl] = {(double)dl[sl].x, (double)dl[sl].y, (double)dl[sl].z};
                const Feature<double> f = fc[k];
                double d1, d2;
                feat_dir_derivs(f, X, dd, d1, d2);
                const Barrier3 bb = barrier_all(d, (double)dh);
                const EdgeMoll em = edge_moll(X, ee_eps(D, M, E, q.x, gsl, isl));
                acc += kap * moll_barrier_dir2(em, dd, d1, d2, bb);
                bv = em.m * bb.b;
            }
        } else {
            V3<float> Xf[4];
            load_slots<float>(D, P, M, gsl, isl, 0.0f, s, Xf);
            Feature<float> f = pair_feature<float>(q.x, Xf);
            d = f.d;
            if (d < dh) {
                float d1, d2;
                feat_dir_derivs(f, Xf, dl, d1, d2);
                const Barrier3T<float> bb = barrier_all(d, dh);
                const EdgeMollT<float> em = edge_moll(Xf, (float)ee_eps(D, M, E, q.x, gsl, isl));
                acc += kap * moll_barrier_dir2(em, dl, d1, d2, bb);
                bv = (double)(em.m * bb.b);
            }
        }
        bcur[k] = bv;
        if (pk > 0.f) amin = fmin(amin, R(kEta) * d / R(pk));
    }
    // friction (lagged pairs)
    const LagRec* lg = D.lag + P.pair_off;
    if (P.mu_f > 0.f)
        for (int l = threadIdx.x; l < nl; l += kThreads) {
            const LagRec& L = lg[l];
            R Dl[3] = {R(-s * L.dY[0]), R(-s * L.dY[1]), R(-s * L.dY[2])}, pd[3] = {R(0), R(0), R(0)};
            for (int gs = 0; gs < 3; ++gs)
                if (L.g[gs] >= 0) {
                    int si = P.v_off + L.g[gs];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        int sc = c * D.Vt + si;
                        Dl[c] += R(L.w[gs]) * R((D.uh[sc] - D.u0h[sc]) + (D.ul[sc] - D.u0l[sc]));
                        pd[c] += R(L.w[gs]) * R(D.p[sc]);
                    }
                }
            R nD = L.n[0] * Dl[0] + L.n[1] * Dl[1] + L.n[2] * Dl[2];
            R np_ = L.n[0] * pd[0] + L.n[1] * pd[1] + L.n[2] * pd[2];
            R tD[3], tp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                tD[c] = Dl[c] - L.n[c] * nD;
                tp[c] = pd[c] - L.n[c] * np_;
            }
            R sv = sqrt(tD[0] * tD[0] + tD[1] * tD[1] + tD[2] * tD[2]);
            R eps = P.eps_v, cf = R(P.mu_f) * R(L.lam);
            R tp2 = tp[0] * tp[0] + tp[1] * tp[1] + tp[2] * tp[2];
            R up = sv > R(0) ? (tD[0] * tp[0] + tD[1] * tp[1] + tD[2] * tp[2]) / sv : R(0);
            acc += cf * (moll_f1_over_s(sv, eps) * tp2 - moll_c(sv, eps) * up * up);
        }
    R v[1] = {acc};
    block_sum_r<R, 1>(v);
    php = (double)v[0];
    if constexpr (kMixed) {
        accd = block_min_d(amin);
    } else {
        float m[1] = {-amin};
        block_max_f<1>(m);
        accd = (double)(-m[0]);
    }
}

// trial pass over pairs at u + alpha p: slot contributions and remainders.
// With alpha > 0 the remainder of pair k subtracts from its barrier value at
// the current point, stored by pair_php of this point; alpha = 0 evaluates
// the current point itself (remainder 0) and needs no stored value.
template <typename R>
__device__ __noinline__ void pair_trial(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np, int nl, double s,
                           float alpha, double& rem, int& bad, float& fsc) {
    constexpr bool kMixed = sizeof(R) == 8;   // float64 features; else the plain-FP32 form
    R acc = R(0);
    int badl = 0;
    float fm = 0.f;   // largest slot force component written (float32 resolution scale)
    const int4* pr = D.pairs + P.pair_off;
    const double* bcur = D.bpair + P.pair_off;
    Feature<double>* fc = D.fcache + P.pair_off;
    float* sb = D.slotbuf + (size_t)9 * 6 * P.pair_off;
    const R dh = P.dhat, kap = P.kappa;
    const bool trial = alpha != 0.0f;
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        V3<float> Xf[4];
        load_slots<float>(D, P, M, gsl, isl, alpha, s, Xf);
        int mask = 31;
        float d1f;
        if constexpr (kMixed)
            d1f = pair_pick(q.x, Xf, mask);
        else
            d1f = pair_feature<float>(q.x, Xf).d;
        const R b0 = trial ? R(bcur[k]) : R(0);
        float out[3][9];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 9; ++c) out[a][c] = 0.f;
        if (kMixed && (double)d1f > kNearBand * (double)dh) {
            acc += kap * b0;                    // b = 0 at the trial point
            fc[k].nf = -1;
            fc[k].d = (double)d1f * (1.0 - 1e-5);
        } else {
            V3<R> X1[4];
            Feature<R> f1;
            if constexpr (kMixed) {
                load_slots<double>(D, P, M, gsl, isl, alpha, s, X1);
                f1 = pair_feature<double>(q.x, X1, mask);
                fc[k] = f1;
            } else {
#pragma unroll
                for (int sl = 0; sl < 4; ++sl) X1[sl] = Xf[sl];
                f1 = pair_feature<float>(q.x, X1);
            }
            if (!(f1.d > R(0))) {
                badl = 1;
            } else if (f1.d >= dh) {
                acc += kap * b0;
            } else {
                V3<R> r = feat_r(f1, X1);
                R inv = R(1) / f1.d;
                V3<R> rh = inv * r;
                const Barrier3T<R> bb = barrier_all(f1.d, dh);
                const EdgeMollT<R> em = edge_moll(X1, R(ee_eps(D, M, E, q.x, gsl, isl)));
                // gradient of m(c) b(d): m b' w_s r^ + m' b dc/dX_s; Gauss-Newton
                // block m b'' w_s^2 r^ r^T (a preconditioner entry: float32)
                R b1 = kap * em.m * bb.b1, b2 = kap * em.m * bb.b2, cb = kap * em.m1 * bb.b;
                const float rx = (float)rh.x, ry = (float)rh.y, rz = (float)rh.z;
                R gdp = R(0);
#pragma unroll
                for (int sl = 0; sl < 3; ++sl)
                    if (gsl[sl] >= 0) {
                        int si = P.v_off + gsl[sl];
                        V3<R> pv = {R(D.p[si]), R(D.p[D.Vt + si]), R(D.p[2 * D.Vt + si])};
                        V3<R> gs = (b1 * f1.w[sl]) * rh;
                        if (em.on) gs = gs + cb * edge_moll_grad(em, sl);
                        gdp += dot(gs, pv);
                        const float kw = (float)(b2 * f1.w[sl] * f1.w[sl]);
                        out[sl][0] = (float)gs.x;
                        out[sl][1] = (float)gs.y;
                        out[sl][2] = (float)gs.z;
                        fm = fmaxf(fm, fmaxf(fabsf(out[sl][0]), fmaxf(fabsf(out[sl][1]), fabsf(out[sl][2]))));
                        out[sl][3] = kw * rx * rx;
                        out[sl][4] = kw * ry * ry;
                        out[sl][5] = kw * rz * rz;
                        out[sl][6] = kw * rx * ry;
                        out[sl][7] = kw * rx * rz;
                        out[sl][8] = kw * ry * rz;
                    }
                if (trial) acc += kap * b0 - kap * em.m * bb.b + (R)alpha * gdp;
            }
        }
#pragma unroll
        for (int sl = 0; sl < 3; ++sl)
            if (gsl[sl] >= 0)
#pragma unroll
                for (int c = 0; c < 9; ++c) sb[9 * (3 * k + sl) + c] = out[sl][c];
    }
    const LagRec* lg = D.lag + P.pair_off;
    for (int l = threadIdx.x; l < nl; l += kThreads) {
        const LagRec& L = lg[l];
        R D1[3] = {R(-s * L.dY[0]), R(-s * L.dY[1]), R(-s * L.dY[2])}, pd[3] = {R(0), R(0), R(0)};
        for (int gs = 0; gs < 3; ++gs)
            if (L.g[gs] >= 0) {
                int si = P.v_off + L.g[gs];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int sc = c * D.Vt + si;
                    float pv = D.p[sc];
                    D1[c] += (R)L.w[gs] * (R)((D.uh[sc] - D.u0h[sc]) + (D.ul[sc] - D.u0l[sc]) + alpha * pv);
                    pd[c] += (R)L.w[gs] * (R)pv;
                }
            }
        R D0[3] = {D1[0] - alpha * pd[0], D1[1] - alpha * pd[1], D1[2] - alpha * pd[2]};
        R n1 = L.n[0] * D1[0] + L.n[1] * D1[1] + L.n[2] * D1[2];
        R n0 = L.n[0] * D0[0] + L.n[1] * D0[1] + L.n[2] * D0[2];
        R t1[3], t0[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            t1[c] = D1[c] - L.n[c] * n1;
            t0[c] = D0[c] - L.n[c] * n0;
        }
        R s1 = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
        R s0 = sqrt(t0[0] * t0[0] + t0[1] * t0[1] + t0[2] * t0[2]);
        R eps = P.eps_v, cf = (R)P.mu_f * (R)L.lam;
        R f1s = moll_f1_over_s(s1, eps), cs = moll_c(s1, eps);
        R tdp = t1[0] * pd[0] + t1[1] * pd[1] + t1[2] * pd[2];
        acc += cf * (moll_f(s0, eps) - moll_f(s1, eps) + (R)alpha * f1s * tdp);
        R uh[3] = {0, 0, 0};
        if (s1 > 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) uh[c] = t1[c] / s1;
        // tangent-plane Hessian f'/s (I - n n^T) - c(s) u u^T
        R Hn[6];
        Hn[0] = f1s * (R(1) - L.n[0] * L.n[0]) - cs * uh[0] * uh[0];
        Hn[1] = f1s * (R(1) - L.n[1] * L.n[1]) - cs * uh[1] * uh[1];
        Hn[2] = f1s * (R(1) - L.n[2] * L.n[2]) - cs * uh[2] * uh[2];
        Hn[3] = -f1s * L.n[0] * L.n[1] - cs * uh[0] * uh[1];
        Hn[4] = -f1s * L.n[0] * L.n[2] - cs * uh[0] * uh[2];
        Hn[5] = -f1s * L.n[1] * L.n[2] - cs * uh[1] * uh[2];
        for (int gs = 0; gs < 3; ++gs)
            if (L.g[gs] >= 0) {
                float* e = sb + 9 * (3 * (P.pair_cap + l) + gs);
                R gw = cf * f1s * L.w[gs], kw = cf * L.w[gs] * L.w[gs];
                e[0] = (float)(gw * t1[0]);
                e[1] = (float)(gw * t1[1]);
                e[2] = (float)(gw * t1[2]);
                fm = fmaxf(fm, fmaxf(fabsf(e[0]), fmaxf(fabsf(e[1]), fabsf(e[2]))));
                for (int c = 0; c < 6; ++c) e[3 + c] = (float)(kw * Hn[c]);
            }
    }
    // the features just written are those of the point the caller continues
    // from when this trial is accepted (or of the current point, alpha = 0)
    if (threadIdx.x == 0) S.fok = kMixed ? 1 : 0;
    R v[1] = {acc};
    block_sum_r<R, 1>(v);
    rem = (double)v[0];
    float fmv[1] = {fm};
    block_max_f<1>(fmv);
    fsc = fmv[0];
    if (badl) S.flag = 1;
    __syncthreads();
    bad = S.flag;
    __syncthreads();
    if (threadIdx.x == 0) S.flag = 0;
    __syncthreads();
}

// lag records: candidates closer than dhat at the frame start
template <typename R>
__device__ __noinline__ int lag_build(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np) {
    const int4* pr = D.pairs + P.pair_off;
    LagRec* lg = D.lag + P.pair_off;
    const double dh = P.dhat, kap = P.kappa;
    int run = 0;
    for (int b0 = 0; b0 < np; b0 += kThreads) {
        int k = b0 + threadIdx.x;
        int keep = 0;
        LagRec L;
        if (k < np && P.mu_f > 0.f) {
            int gsl[4], isl[4];
            int4 q = pr[k];
            pair_slots(D, M, E, q, gsl, isl);
            V3<R> X[4];
            load_slots<R>(D, P, M, gsl, isl, 0.0f, 0.0, X);
            Feature<R> f = pair_feature<R>(q.x, X);
            if (f.d < R(dh) && f.d > R(0)) {
                keep = 1;
                L.pq[0] = q.x;
                L.pq[1] = q.y;
                L.pq[2] = q.z;
                V3<R> r = feat_r(f, X);
                R inv = R(1) / f.d;
                L.n[0] = (float)(r.x * inv);
                L.n[1] = (float)(r.y * inv);
                L.n[2] = (float)(r.z * inv);
                L.lam = (double)(-R(kap) * edge_moll(X, R(ee_eps(D, M, E, q.x, gsl, isl))).m *
                                 barrier_all(f.d, R(dh)).b1);
                R dY[3] = {0, 0, 0};
                int ni = 0;
                for (int q = 0; q < 3; ++q) {
                    L.iv[q] = -1;
                    L.iw[q] = 0.f;
                }
                for (int sl = 0; sl < 4; ++sl) {
                    if (sl < 3) {
                        L.g[sl] = gsl[sl];          // mesh-local vertex id or -1
                        L.w[sl] = gsl[sl] >= 0 ? (float)f.w[sl] : 0.f;
                    }
                    if (isl[sl] >= 0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            dY[c] += -f.w[sl] * ((R)D.Yn[3 * (P.yw_off + isl[sl]) + c] -
                                                 (R)D.Yt[3 * (P.yw_off + isl[sl]) + c]);
                        if (ni < 3) {
                            L.iv[ni] = isl[sl];
                            L.iw[ni] = (float)(-f.w[sl]);
                            ++ni;
                        }
                    }
                }
                L.dY[0] = (float)dY[0];
                L.dY[1] = (float)dY[1];
                L.dY[2] = (float)dY[2];
            }
        }
        int tot;
        int pos = block_scan(keep, tot) + run;
        if (keep) lg[pos] = L;
        run += tot;
    }
    __syncthreads();
    return run;
}

// ---------------------------------------------------------------------------
// vertex passes

struct Dots {
    double zy, yPy, pg1, yp;
    float ginf;
    int bad;
};

// Completes g and the blocks at u + alpha p (inertia, Dirichlet), applies
// the preconditioner and reduces the Dai-Kou dot products.
// The vertex passes issue every load of two vertices before any store or
// branch (the Dirichlet flag is read as a value), so that each thread keeps
// its memory requests in flight together; vertices are visited in the same
// per-thread order (i, i + kThreads, ...) as a one-by-one loop, so the sums
// do not change.
constexpr int kVertUnroll = 2;

__device__ __noinline__ Dots finalize(const Dev& D, const PadDev& P, const MeshDev& M, float alpha, int gb, int go, bool dots) {
    FSum sv[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    float gi[1] = {0.f};
    int bad = 0;
    const float rho = P.rho;
    // pointers of the pad's state, read once (see TetPtrs)
    const size_t Vt = D.Vt;
    float* g = D.g[gb] + P.v_off;
    const float* gold = D.g[go] + P.v_off;
    const float* blk = D.blk[gb] + P.v_off;
    const float* uhp = D.uh + P.v_off;
    const float* ulp = D.ul + P.v_off;
    const float* uhatp = D.uhat + P.v_off;
    const float* pp = D.p + P.v_off;
    float* zp = D.z + P.v_off;
    const uint8_t* fxp = D.fixed + M.xv_off;
    const float* vlp = D.vlump + M.xv_off;
    const int n_v = M.n_v;
    const bool blockp = P.precond == 0;
    const bool plain = P.prec != 0;          // plain-FP32 form: float sums
    for (int i0 = threadIdx.x; i0 < n_v; i0 += kVertUnroll * kThreads) {
        float mm[kVertUnroll], pv[kVertUnroll][3], du[kVertUnroll][3], gg[kVertUnroll][3], go3[kVertUnroll][3];
        float K[kVertUnroll][6];
        bool fx[kVertUnroll], ok[kVertUnroll];
#pragma unroll
        for (int u = 0; u < kVertUnroll; ++u) {
            const int i = i0 + u * kThreads;
            ok[u] = i < n_v;
            const int ii = ok[u] ? i : i0;             // in-bounds index for the loads
            fx[u] = fxp[ii] != 0;
            mm[u] = rho * vlp[ii];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t sc = c * Vt + ii;
                pv[u][c] = pp[sc];
                du[u][c] = (uhp[sc] - uhatp[sc]) + ulp[sc];
                gg[u][c] = g[sc];
                go3[u][c] = dots ? gold[sc] : 0.f;
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) K[u][c] = blk[c * Vt + ii];
        }
#pragma unroll
        for (int u = 0; u < kVertUnroll; ++u) {
            if (!ok[u]) continue;
            const size_t si = (size_t)i0 + u * kThreads;
            if (fx[u]) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    g[c * Vt + si] = 0.f;
                    zp[c * Vt + si] = 0.f;
                }
                continue;
            }
            const float m = mm[u];
            float g1[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                g1[c] = gg[u][c] + m * (du[u][c] + alpha * pv[u][c]);
                g[c * Vt + si] = g1[c];
            }
            float Kv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) Kv[c] = K[u][c];
            Kv[0] += m; Kv[1] += m; Kv[2] += m;
            float Ki[6];
            if (blockp) {
                if (!sym_inverse(Kv, Ki)) bad = 1;
            } else {
                Ki[0] = 1.f / Kv[0]; Ki[1] = 1.f / Kv[1]; Ki[2] = 1.f / Kv[2];
                Ki[3] = Ki[4] = Ki[5] = 0.f;
            }
            float z[3];
            sym_apply(Ki, g1, z);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                zp[c * Vt + si] = z[c];
                gi[0] = fmaxf(gi[0], fabsf(g1[c]));
            }
            if (!(isfinite(g1[0]) && isfinite(g1[1]) && isfinite(g1[2]))) bad = 1;
            if (dots) {
                float y[3], Py[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) y[c] = g1[c] - go3[u][c];
                sym_apply(Ki, y, Py);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    fsum_add_mode(sv[0], __fmul_rn(z[c], y[c]), plain);
                    fsum_add_mode(sv[1], __fmul_rn(y[c], Py[c]), plain);
                    fsum_add_mode(sv[2], __fmul_rn(pv[u][c], g1[c]), plain);
                    fsum_add_mode(sv[3], __fmul_rn(y[c], pv[u][c]), plain);
                }
            }
        }
    }
    if (bad) S.flag = 1;
    double v[4];
    block_sum_fsum<4>(sv, v, plain);
    block_max_f<1>(gi);
    Dots d{v[0], v[1], v[2], v[3], gi[0], 0};
    d.bad = S.flag;
    __syncthreads();
    if (threadIdx.x == 0) S.flag = 0;
    __syncthreads();
    return d;
}

struct DirOut {
    double gTp, pMp;
    float pn;
};

// optionally u += alpha p (double-float), then p = -z + beta p; reduces
// g^T p, p^T M p and max_i |p_i|
__device__ __noinline__ DirOut direction(const Dev& D, const PadDev& P, const MeshDev& M, float alpha, bool move, double beta,
                            int gb) {
    FSum sgp{0.f, 0.f}, smp{0.f, 0.f};
    float pn[1] = {0.f};
    const float rho = P.rho;
    const float bf = (float)beta;
    // pointers of the pad's state, read once (see TetPtrs)
    const size_t Vt = D.Vt;
    const float* g = D.g[gb] + P.v_off;
    float* uhp = D.uh + P.v_off;
    float* ulp = D.ul + P.v_off;
    float* pp = D.p + P.v_off;
    const float* zp = D.z + P.v_off;
    const uint8_t* fxp = D.fixed + M.xv_off;
    const float* vlp = D.vlump + M.xv_off;
    const int n_v = M.n_v;
    const bool plain = P.prec != 0;          // plain-FP32 form: float u, float sums
    for (int i0 = threadIdx.x; i0 < n_v; i0 += kVertUnroll * kThreads) {
        float mm[kVertUnroll], pv[kVertUnroll][3], zv[kVertUnroll][3], gv[kVertUnroll][3];
        float uh[kVertUnroll][3], ul[kVertUnroll][3];
        bool fx[kVertUnroll], ok[kVertUnroll];
#pragma unroll
        for (int u = 0; u < kVertUnroll; ++u) {
            const int i = i0 + u * kThreads;
            ok[u] = i < n_v;
            const int ii = ok[u] ? i : i0;
            fx[u] = fxp[ii] != 0;
            mm[u] = rho * vlp[ii];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t sc = c * Vt + ii;
                pv[u][c] = pp[sc];
                zv[u][c] = zp[sc];
                gv[u][c] = g[sc];
                uh[u][c] = move ? uhp[sc] : 0.f;
                ul[u][c] = move ? ulp[sc] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < kVertUnroll; ++u) {
            if (!ok[u]) continue;
            const size_t si = (size_t)i0 + u * kThreads;
            float n2 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t sc = c * Vt + si;
                if (move && !fx[u]) {
                    // u += alpha p as a double-float sum (hi, lo)
                    float t = alpha * pv[u][c];
                    float hi = uh[u][c], lo = ul[u][c];
                    if (plain) {
                        uhp[sc] = hi + t;
                    } else {
                        float sm = hi + t;
                        float bb = sm - hi;
                        float err = (hi - (sm - bb)) + (t - bb);
                        lo += err;
                        float nh = sm + lo;
                        ulp[sc] = lo - (nh - sm);
                        uhp[sc] = nh;
                    }
                }
                float np = fx[u] ? 0.f : (-zv[u][c] + bf * pv[u][c]);
                pp[sc] = np;
                n2 += np * np;
                fsum_add_mode(sgp, __fmul_rn(gv[u][c], np), plain);
            }
            fsum_add_mode(smp, __fmul_rn(mm[u], n2), plain);
            pn[0] = fmaxf(pn[0], sqrtf(n2));
        }
    }
    const FSum sums[2] = {sgp, smp};
    double v[2];
    block_sum_fsum<2>(sums, v, plain);
    block_max_f<1>(pn);
    return DirOut{v[0], v[1], pn[0]};
}

// p = -P g at the current point from the stored gradient g[gb] (inertia
// included) and blocks blk[gb] (without the mass), for a restart after
// trial points overwrote z; reduces g^T p, p^T M p and max_i |p_i|
__device__ __noinline__ DirOut steepest_direction(const Dev& D, const PadDev& P, const MeshDev& M, int gb) {
    FSum sgp{0.f, 0.f}, smp{0.f, 0.f};
    float pn[1] = {0.f};
    const bool plain = P.prec != 0;
    const size_t Vt = D.Vt;
    const float* g = D.g[gb] + P.v_off;
    const float* blk = D.blk[gb] + P.v_off;
    float* pp = D.p + P.v_off;
    float* zp = D.z + P.v_off;
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        const bool fx = D.fixed[M.xv_off + i] != 0;
        const float m = P.rho * D.vlump[M.xv_off + i];
        float gv[3], K[6], Ki[6], z[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; ++c) gv[c] = g[c * Vt + i];
        if (!fx) {
#pragma unroll
            for (int c = 0; c < 6; ++c) K[c] = blk[c * Vt + i];
            K[0] += m; K[1] += m; K[2] += m;
            if (P.precond == 0) {
                if (sym_inverse(K, Ki)) sym_apply(Ki, gv, z);
            } else {
                z[0] = gv[0] / K[0]; z[1] = gv[1] / K[1]; z[2] = gv[2] / K[2];
            }
        }
        float n2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            zp[c * Vt + i] = z[c];
            pp[c * Vt + i] = -z[c];
            n2 += z[c] * z[c];
            fsum_add_mode(sgp, __fmul_rn(gv[c], -z[c]), plain);
        }
        fsum_add_mode(smp, __fmul_rn(m, n2), plain);
        pn[0] = fmaxf(pn[0], sqrtf(n2));
    }
    const FSum sums[2] = {sgp, smp};
    double v[2];
    block_sum_fsum<2>(sums, v, plain);
    block_max_f<1>(pn);
    return DirOut{v[0], v[1], pn[0]};
}

// Gel motion of an indenter substep per unit of the path parameter s into
// p: the inertial prediction xhat - x^t = h v of Eq. (varopt), zero on
// Dirichlet vertices (the same for every substep of the frame). Returns
// max_i |p_i - c| (the gel part of the advance's motion bound about the
// indenter displacement c).
__device__ __noinline__ float advance_direction(const Dev& D, const PadDev& P, const MeshDev& M, const float c3[3]) {
    float pn[1] = {0.f};
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
        bool fx = D.fixed[M.xv_off + i] != 0;
        float n2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + si;
            float v = fx ? 0.f : P.h * D.vel[sc];
            D.p[sc] = v;
            n2 += (v - c3[c]) * (v - c3[c]);
        }
        pn[0] = fmaxf(pn[0], sqrtf(n2));
    }
    block_max_f<1>(pn);
    return pn[0];
}

// The largest advances of the path parameter that keep every candidate's
// gap above (1 - eta) of itself: bm[0] with the gel moving along p and the
// indenter along Yn - Yt, eta * min_k d_k / max_{i in gel(k), j in ind(k)}
// |p_i - dy_j|, and bm[1] with the gel held (p = 0 in the same bound). Along
// straight motions of both sides, any point of one primitive approaches any
// point of the other at most that fast (both points are convex combinations
// of their primitive's vertices).
template <typename R>
__device__ __noinline__ void pair_advance_bound(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E,
                                                int np, double s, double bm[2]) {
    R bmov = R(3e38), bheld = R(3e38);
    const int4* pr = D.pairs + P.pair_off;
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        float rel = 0.f, rel0 = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (isl[b] < 0) continue;
            const float* yt = D.Yt + 3 * (P.yw_off + isl[b]);
            const float* yn = D.Yn + 3 * (P.yw_off + isl[b]);
            const float y0 = yn[0] - yt[0], y1 = yn[1] - yt[1], y2 = yn[2] - yt[2];
            rel0 = fmaxf(rel0, sqrtf(y0 * y0 + y1 * y1 + y2 * y2));
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (gsl[a] < 0) continue;
                const int si = P.v_off + gsl[a];
                const float e0 = D.p[si] - y0, e1 = D.p[D.Vt + si] - y1, e2 = D.p[2 * D.Vt + si] - y2;
                rel = fmaxf(rel, sqrtf(e0 * e0 + e1 * e1 + e2 * e2));
            }
        }
        if (rel > 0.f || rel0 > 0.f) {
            const R d = pair_distance<R>(D, P, M, q.x, gsl, isl, 0.0f, s, kNearBand * P.dhat);
            if (rel > 0.f) bmov = fmin(bmov, R(kEta) * d / (R(rel) * R(1.0 + 1e-6)));
            if (rel0 > 0.f) bheld = fmin(bheld, R(kEta) * d / (R(rel0) * R(1.0 + 1e-6)));
        }
    }
    if constexpr (sizeof(R) == 8) {
        bm[0] = block_min_d(bmov);
        bm[1] = block_min_d(bheld);
    } else {
        float m[2] = {-bmov, -bheld};
        block_max_f<2>(m);
        bm[0] = (double)(-m[0]);
        bm[1] = (double)(-m[1]);
    }
}

// The pair passes in the pad's precision form: float64 features, barrier,
// step bounds and sums (precision_mode 0), or all float32 (1, the plain form)
__device__ __forceinline__ int lag_build_p(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np) {
    return P.prec ? lag_build<float>(D, P, M, E, np) : lag_build<double>(D, P, M, E, np);
}
__device__ __forceinline__ void pair_php_p(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np,
                                           int nl, double s, double& php, double& accd) {
    if (P.prec)
        pair_php<float>(D, P, M, E, np, nl, s, php, accd);
    else
        pair_php<double>(D, P, M, E, np, nl, s, php, accd);
}
__device__ __forceinline__ void pair_trial_p(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np,
                                             int nl, double s, float alpha, double& rem, int& bad, float& fsc) {
    if (P.prec)
        pair_trial<float>(D, P, M, E, np, nl, s, alpha, rem, bad, fsc);
    else
        pair_trial<double>(D, P, M, E, np, nl, s, alpha, rem, bad, fsc);
}
__device__ __forceinline__ void pair_advance_bound_p(const Dev& D, const PadDev& P, const MeshDev& M,
                                                     const EnvDev& E, int np, double s, double bm[2]) {
    if (P.prec)
        pair_advance_bound<float>(D, P, M, E, np, s, bm);
    else
        pair_advance_bound<double>(D, P, M, E, np, s, bm);
}

// ---------------------------------------------------------------------------
// frame setup: indenter world vertices, u0 = u, uhat = u + h v

__device__ void rotation_dd(const double* pose, double R[9]) {
    double rx = pose[0], ry = pose[1], rz = pose[2];
    double th = sqrt(rx * rx + ry * ry + rz * rz);
    double kx = 0, ky = 0, kz = 0, sn = 0, cs1 = 0;
    if (th > 1e-300) {
        kx = rx / th; ky = ry / th; kz = rz / th;
        sn = sin(th);
        cs1 = 1.0 - cos(th);
    }
    double K[9] = {0, -kz, ky, kz, 0, -kx, -ky, kx, 0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double kk = 0;
            for (int k = 0; k < 3; ++k) kk += K[3 * i + k] * K[3 * k + j];
            R[3 * i + j] = (i == j ? 1.0 : 0.0) + sn * K[3 * i + j] + cs1 * kk;
        }
}

__device__ void rotation(const float* pose, double R[9]) {
    const double r[3] = {pose[0], pose[1], pose[2]};
    rotation_dd(r, R);
}

__device__ __noinline__ void world_indenter(const Dev& D, const PadDev& P, const EnvDev& E, const float* pose, float* Yw) {
    double R[9];
    rotation(pose, R);
    for (int j = threadIdx.x; j < E.n_v; j += kThreads) {
        const float* y = D.Y + 3 * (E.y_off + j);
        for (int c = 0; c < 3; ++c)
            Yw[3 * (P.yw_off + j) + c] =
                (float)(R[3 * c] * y[0] + R[3 * c + 1] * y[1] + R[3 * c + 2] * y[2] + (double)pose[3 + c]);
    }
}

// ---------------------------------------------------------------------------
// the frame solve of one pad

enum { ST_CONVERGED = 0, ST_MAXITER = 1, ST_NONFINITE = 2, ST_LINESEARCH = 3, ST_OVERFLOW = 4 };

struct PadCounters {
    long long iters, substeps, rebuilds, halvings, tet_passes, vert_passes, pair_evals, peak_pairs;
};

__device__ void solve_pad(const Dev& D, int pad) {
    load_pad(D, pad);
    const PadDev& P = S.P;
    const MeshDev& M = S.M;
    const EnvDev& E = S.E;
    const int tid = threadIdx.x;
    PadCounters ctr{0, 0, 0, 0, 0, 0, 0, 0};
    int status = ST_CONVERGED;
    unsigned long long t0 = 0;
    if (tid == 0) t0 = global_ns();
    PhaseClock clk;
    clk.start();
    // frame setup
    world_indenter(D, P, E, D.pose_t + 6 * pad, D.Yt);
    world_indenter(D, P, E, D.pose_n + 6 * pad, D.Yn);
    for (int i = tid; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + si;
            float hi = D.uh[sc], lo = D.ul[sc];
            D.u0h[sc] = hi;
            D.u0l[sc] = lo;
            D.uhat[sc] = (hi + lo) + P.h * D.vel[sc];
        }
    }
    __syncthreads();
    // indenter displacement dy_j = Yn_j - Yt_j over the frame: its largest
    // norm and its spread max_j |dy_j - dy_0| about vertex 0's enter the
    // advance's motion bounds
    float dy0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) dy0[c] = D.Yn[3 * P.yw_off + c] - D.Yt[3 * P.yw_off + c];
    float dyv[2] = {0.f, 0.f};
    for (int j = tid; j < E.n_v; j += kThreads) {
        float a = 0.f, b = 0.f;
        for (int c = 0; c < 3; ++c) {
            float d = D.Yn[3 * (P.yw_off + j) + c] - D.Yt[3 * (P.yw_off + j) + c];
            a += d * d;
            b += (d - dy0[c]) * (d - dy0[c]);
        }
        dyv[0] = fmaxf(dyv[0], sqrtf(a));
        dyv[1] = fmaxf(dyv[1], sqrtf(b));
    }
    block_max_f<2>(dyv);
    const double Dy = (double)dyv[0] * (1.0 + 1e-6), Dspread = (double)dyv[1];
    const double dh = P.dhat, margin = P.dhat;
    const double rbp = (dh + margin) * (1.0 + 1e-6);
    int4* pairs = D.pairs + P.pair_off;
    int* il = D.ilist + P.il_off;
    double s = 0.0, Mb = 0.0;
    ContactCtl cc{0, 0, 0};
    {
        SrcState src{&D, &P, &M, 0.0f};
        int n = bp_build(src, D, M, E, il, rbp, pairs, P.pair_cap);
        ctr.rebuilds++;
        ctr.peak_pairs = n;
        if (n > P.pair_cap) status = ST_OVERFLOW;
        cc.npairs = min(n, P.pair_cap);
    }
    if (status == ST_CONVERGED) {
        cc.nlag = lag_build_p(D, P, M, E, cc.npairs);
        csr_build(D, P, M, E, cc);
    }
    clk.lap(PH_SETUP);
    float g_ref = P.g_ref;   // becomes max(floor, |g| after the first substep)
    bool have_ref = false;
    float fmax = 0.f;        // force scale of the float32 resolution floor: the largest force
                             // component summed into the float32 gradient (elastic corner,
                             // barrier and friction slot forces)
    float target = 0.f;
    int gc = 0;              // buffer holding the current gradient
    float ginf = 0.f;
    while (status == ST_CONVERGED) {
        // advance the indenter and the gel together by ds of the path: the
        // gel along its predicted motion (p) or held, whichever the per-pair
        // bound lets go further (every candidate's gap stays above (1 - eta)
        // of itself). The motion bound of a moving advance is
        // max_j |dy_j - dy_0| + max_i |p_i - dy_0|
        const double Bmov = (Dspread + (double)advance_direction(D, P, M, dy0)) * (1.0 + 1e-6);
        double bnd[2];
        pair_advance_bound_p(D, P, M, E, cc.npairs, s, bnd);
        ctr.pair_evals += cc.npairs;
        double cap_m = 1e300, cap_h = 1e300;
        bool moving = fmin(1.0 - s, bnd[0]) >= fmin(1.0 - s, bnd[1]);
        double ds = fmin(1.0 - s, moving ? bnd[0] : bnd[1]);
        double B = moving ? Bmov : Dy;
        if (Mb + ds * B > margin) {
            SrcState src{&D, &P, &M, (float)s};
            int n = bp_build(src, D, M, E, il, rbp, pairs, P.pair_cap);
            ctr.rebuilds++;
            ctr.peak_pairs = max(ctr.peak_pairs, (long long)n);
            if (n > P.pair_cap) { status = ST_OVERFLOW; break; }
            cc.npairs = n;
            csr_build(D, P, M, E, cc);
            Mb = 0.0;
            pair_advance_bound_p(D, P, M, E, cc.npairs, s, bnd);
            ctr.pair_evals += cc.npairs;
            if (Bmov > 0.0) cap_m = margin / Bmov;
            if (Dy > 0.0) cap_h = margin / Dy;
            const double dm = fmin(fmin(1.0 - s, bnd[0]), cap_m), dhl = fmin(fmin(1.0 - s, bnd[1]), cap_h);
            moving = dm >= dhl;
            ds = moving ? dm : dhl;
            B = moving ? Bmov : Dy;
        }
        const float am = moving ? 1.0f : 0.0f;   // the gel's share of the advance
        clk.lap(PH_BROAD);
        // the gradient at the advanced state; ds halves while that state
        // leaves E's domain (an inverted tet)
        const int gn = gc ^ 1;
        bool ok = false;
        double s1 = s;
        TetOut to{};
        Dots d0{};
        float fsc0 = 0.f;
        for (int hv = 0; hv <= kMaxHalvings; ++hv) {
            s1 = (ds >= 1.0 - s) ? 1.0 : s + ds;
            const float ag = am * (float)ds;
            to = tet_pass<1>(D, P, M, ag, gn);
            ctr.tet_passes++;
            clk.lap(PH_TET1);
            double rem0;
            int badp;
            pair_trial_p(D, P, M, E, cc.npairs, cc.nlag, s1, ag, rem0, badp, fsc0);
            ctr.pair_evals += cc.npairs;
            contact_gather(D, P, cc, gn);
            clk.lap(PH_PAIR_TRIAL);
            d0 = finalize(D, P, M, ag, gn, gc, false);
            ctr.vert_passes++;
            clk.lap(PH_VERTEX);
            if (!to.bad && !badp && !d0.bad) {
                ok = true;
                break;
            }
            ds *= 0.5;
        }
        if (!ok) { status = ST_NONFINITE; break; }
        // u += ds p (gel moving), then p = -P g at the advanced state
        DirOut dir = direction(D, P, M, am * (float)ds, moving, 0.0, gn);
        ctr.vert_passes++;
        clk.lap(PH_VERTEX);
        gc = gn;
        s = s1;
        Mb += ds * B;
        ctr.substeps++;
        ginf = d0.ginf;
        fmax = fmaxf(to.fmax, fsc0);
        if (!have_ref) {
            g_ref = fmaxf(g_ref, ginf);
            have_ref = true;
        }
        const float rel = (s >= 1.0) ? P.tol : fmaxf(P.tol, P.tol_adv);
        target = fmaxf(rel * g_ref, P.floor * fmax);
        bool retried = false;
        while (ginf > target && ctr.iters < P.max_iter) {
            if (dir.pn == 0.f || dir.gTp >= 0.0) {
                dir = direction(D, P, M, 0.0f, false, 0.0, gc);
                ctr.vert_passes++;
                if (dir.pn == 0.f) break;
            }
            double a_up = dh / (2.0 * (double)dir.pn);
            clk.lap(PH_VERTEX);
            TetOut tp = tet_pass<0>(D, P, M, 0.0f, gc);
            ctr.tet_passes++;
            clk.lap(PH_TET0);
            double php_c, a_ccd;
            pair_php_p(D, P, M, E, cc.npairs, cc.nlag, s, php_c, a_ccd);
            ctr.pair_evals += cc.npairs;
            clk.lap(PH_PAIR_PHP);
            double pHp = tp.acc + php_c + dir.pMp;
            double a_bar = pHp > 0.0 ? -dir.gTp / pHp : 1e300;
            const bool literal = P.step == 1;   // Eq. (step_size) as printed: no CCD bound
            if (literal) a_ccd = 1e300;
            double alpha = fmin(fmin(a_up, a_ccd), a_bar);
            if (Mb + alpha * dir.pn > margin) {
                SrcState src{&D, &P, &M, (float)s};
                int n = bp_build(src, D, M, E, il, rbp, pairs, P.pair_cap);
                ctr.rebuilds++;
                ctr.peak_pairs = max(ctr.peak_pairs, (long long)n);
                if (n > P.pair_cap) { status = ST_OVERFLOW; break; }
                cc.npairs = n;
                csr_build(D, P, M, E, cc);
                Mb = 0.0;
                double dummy;
                pair_php_p(D, P, M, E, cc.npairs, cc.nlag, s, dummy, a_ccd);
                ctr.pair_evals += cc.npairs;
                if (literal) a_ccd = 1e300;
                alpha = fmin(fmin(a_up, a_ccd), a_bar);
                clk.lap(PH_BROAD);
            }
            const int gt = gc ^ 1;
            bool accepted = false;
            Dots dt{};
            for (int hv = 0; hv <= kMaxHalvings; ++hv) {
                float af = (float)alpha;
                TetOut tt = tet_pass<1>(D, P, M, af, gt);
                ctr.tet_passes++;
                clk.lap(PH_TET1);
                double remc;
                int bp;
                float fsc;
                pair_trial_p(D, P, M, E, cc.npairs, cc.nlag, s, af, remc, bp, fsc);
                ctr.pair_evals += cc.npairs;
                contact_gather(D, P, cc, gt);
                clk.lap(PH_PAIR_TRIAL);
                dt = finalize(D, P, M, af, gt, gc, true);
                ctr.vert_passes++;
                clk.lap(PH_VERTEX);
                if (!tt.bad && !bp && !dt.bad) {
                    double a = (double)af;
                    double R = tt.acc + remc + 0.5 * a * a * dir.pMp;
                    double dE = a * dt.pg1 - R;
                    // the literal rule takes any trial state inside E's domain
                    if (literal || dE <= kArmijoC * a * dir.gTp) {
                        accepted = true;
                        alpha = a;
                        fmax = fmaxf(tt.fmax, fsc);
                        break;
                    }
                }
                alpha *= 0.5;
                ctr.halvings++;
            }
            if (!accepted) {
                // one retry along the preconditioned steepest descent -P g
                // before the line search counts as failed
                if (!retried && !literal) {
                    retried = true;
                    if (tid == 0) S.fok = 0;   // the cached features are the last rejected trial's
                    dir = steepest_direction(D, P, M, gc);
                    ctr.vert_passes++;
                    continue;
                }
                status = ST_LINESEARCH;
                break;
            }
            retried = false;
            Mb += alpha * dir.pn;
            ctr.iters++;
            double beta = 0.0;
            if (fabs(dt.yp) > 1e-300) beta = dt.zy / dt.yp - (dt.yPy / dt.yp) * (dt.pg1 / dt.yp);
            dir = direction(D, P, M, (float)alpha, true, beta, gt);
            ctr.vert_passes++;
            if (dir.gTp >= 0.0) {
                dir = direction(D, P, M, 0.0f, false, 0.0, gt);
                ctr.vert_passes++;
            }
            clk.lap(PH_VERTEX);
            gc = gt;
            ginf = dt.ginf;
            target = fmaxf(rel * g_ref, P.floor * fmax);
        }
        if (status != ST_CONVERGED) break;
        if (s >= 1.0) {
            if (ginf > target) status = ST_MAXITER;
            break;
        }
        if (ctr.substeps >= kMaxSubsteps || ctr.iters >= P.max_iter) {
            status = ST_MAXITER;
            break;
        }
    }
    // the current gradient must sit in buffer 0 for the next frame's readers
    // (none today); velocities and pose
    for (int i = tid; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + si;
            D.vel[sc] = ((D.uh[sc] - D.u0h[sc]) + (D.ul[sc] - D.u0l[sc])) / P.h;
        }
    }
    if (tid == 0) {
        if (D.status) D.status[pad] = status;
        if (D.iters) D.iters[pad] = (int)ctr.iters;
        long long* st = D.stats + 16 * pad;
        st[0] = ctr.iters; st[1] = ctr.substeps; st[2] = ctr.rebuilds; st[3] = ctr.halvings;
        st[4] = ctr.tet_passes; st[5] = ctr.vert_passes; st[6] = ctr.pair_evals; st[7] = ctr.peak_pairs;
        clk.lap(PH_VERTEX);
        for (int q = 0; q < PH_COUNT; ++q) st[8 + q] = (long long)clk.acc[q];
        st[15] = (long long)(global_ns() - t0);
        double* nr = D.norms + 4 * pad;
        nr[0] = ginf; nr[1] = target; nr[2] = g_ref; nr[3] = fmax;
        D.pad_nlag[pad] = cc.nlag;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads, kCtasPerSm) solve_kernel(const __grid_constant__ Dev D) {
    if (threadIdx.x == 0) S.flag = 0;
    for (;;) {
        if (threadIdx.x == 0) S.pad = atomicAdd(D.queue, 1);
        __syncthreads();
        int q = S.pad;
        __syncthreads();
        if (q >= D.n_pads) break;
        solve_pad(D, D.order[q]);
    }
}

#ifndef TAC_WIDE
// ---------------------------------------------------------------------------
// processing order of the next solve launch: longest predicted pad first.
// The prediction is the pad's solve time in its previous frame (0 before its
// first frame), the tet count breaking ties, so the first frame runs the
// largest meshes first. One CTA sorts (key descending, pad ascending) with a
// bitonic network over n2 = next power of two >= n_pads entries of global
// scratch; the padding entries (key 0, index INT_MAX) sort last.

__device__ __forceinline__ bool sched_before(unsigned long long ka, int ia, unsigned long long kb, int ib) {
    return ka > kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(1024) schedule_kernel(const __grid_constant__ Dev D, unsigned long long* key,
                                                        int* idx, int n2, int* order) {
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        if (i < D.n_pads) {
            long long ns = D.stats[16 * (size_t)i + 15];
            unsigned long long t = ns > 0 ? (unsigned long long)ns : 0ull;
            t = t < (1ull << 40) ? t : (1ull << 40) - 1;
            int nt = D.meshes[D.pads[i].mesh].n_t;
            key[i] = (t << 22) | (unsigned long long)min(nt, (1 << 22) - 1);
            idx[i] = i;
        } else {
            key[i] = 0ull;
            idx[i] = 0x7fffffff;
        }
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    unsigned long long ki = key[i], kl = key[l];
                    int ii = idx[i], il = idx[l];
                    bool up = (i & k) == 0;
                    bool swap = up ? sched_before(kl, il, ki, ii) : sched_before(ki, ii, kl, il);
                    if (swap) {
                        key[i] = kl; key[l] = ki;
                        idx[i] = il; idx[l] = ii;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < D.n_pads; i += blockDim.x) order[i] = idx[i];
}

// ---------------------------------------------------------------------------
// verification kernel: one CTA per pad (see tac_debug_eval)

__global__ void __launch_bounds__(kThreads) debug_eval_kernel(const __grid_constant__ Dev D, float alpha, double r, float* grad_out,
                                                              float* blk_out, double* scal) {
    if (threadIdx.x == 0) S.flag = 0;
    __syncthreads();
    const int pad = blockIdx.x;
    load_pad(D, pad);
    const PadDev& P = S.P;
    const MeshDev& M = S.M;
    const EnvDev& E = S.E;
    world_indenter(D, P, E, D.pose_t + 6 * pad, D.Yt);
    world_indenter(D, P, E, D.pose_t + 6 * pad, D.Yn);
    __syncthreads();
    SrcState src{&D, &P, &M, 1.0f};
    int n = bp_build(src, D, M, E, D.ilist + P.il_off, r, D.pairs + P.pair_off, P.pair_cap);
    ContactCtl cc{min(n, P.pair_cap), 0, 0};
    csr_build(D, P, M, E, cc);
    // u0 = uhat = u (no inertia offset, no friction lag)
    for (int i = threadIdx.x; i < M.n_v; i += kThreads)
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + P.v_off + i;
            D.u0h[sc] = D.uh[sc];
            D.u0l[sc] = D.ul[sc];
            D.uhat[sc] = D.uh[sc] + D.ul[sc];
        }
    __syncthreads();
    double dmin = pair_dmin(D, P, M, E, cc.npairs, 1.0);
    TetOut tp = tet_pass<0>(D, P, M, 0.0f, 0);
    double php_c, a_ccd;
    pair_php_p(D, P, M, E, cc.npairs, 0, 1.0, php_c, a_ccd);
    double pMp = 0.0;
    {
        double v[1] = {0.0};
        for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
            if (D.fixed[M.xv_off + i]) continue;
            float m = P.rho * D.vlump[M.xv_off + i];
            for (int c = 0; c < 3; ++c) {
                float pv = D.p[c * D.Vt + P.v_off + i];
                v[0] += (double)(m * pv * pv);
            }
        }
        block_sum<1>(v);
        pMp = v[0];
    }
    TetOut tt = tet_pass<1>(D, P, M, alpha, 0);
    double remc;
    int bp;
    float fsc;
    pair_trial_p(D, P, M, E, cc.npairs, 0, 1.0, alpha, remc, bp, fsc);
    contact_gather(D, P, cc, 0);
    // outputs before inertia / inversion: gradient with inertia m alpha p
    double gp[1] = {0.0};
    float gi[1] = {0.f};
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
        int ui = P.v_off + D.vuser[M.xv_off + i];     // output row: input vertex order
        bool fx = D.fixed[M.xv_off + i] != 0;
        float m = P.rho * D.vlump[M.xv_off + i];
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + si;
            float gv = fx ? 0.f : D.g[0][sc] + m * alpha * D.p[sc];
            if (grad_out) grad_out[3 * ui + c] = gv;
            gp[0] += (double)(gv * D.p[sc]);
            gi[0] = fmaxf(gi[0], fabsf(gv));
        }
        if (blk_out)
            for (int c = 0; c < 6; ++c) blk_out[6 * ui + c] = D.blk[0][c * D.Vt + si] + (c < 3 ? m : 0.f);
    }
    block_sum<1>(gp);
    block_max_f<1>(gi);
    if (threadIdx.x == 0 && scal) {
        double a = alpha;
        double R = tt.acc + remc + 0.5 * a * a * pMp;
        double* o = scal + 8 * pad;
        o[0] = tp.acc;
        o[1] = php_c;
        o[2] = pMp;
        o[3] = a * gp[0] - R;
        o[4] = a_ccd;
        o[5] = dmin;
        o[6] = (double)n;
        o[7] = (double)gi[0];
    }
}

// candidate set of one pad for caller positions (see tac_broadphase)
__global__ void __launch_bounds__(kThreads) broadphase_kernel(const __grid_constant__ Dev D, int pad, const float* x, const float* y,
                                                              double r, int* out, int cap, int* count) {
    load_pad(D, pad);
    const PadDev& P = S.P;
    const MeshDev& M = S.M;
    const EnvDev& E = S.E;
    SrcArrays src{x, y, D.vuser + M.xv_off};
    int n = bp_build(src, D, M, E, D.ilist + P.il_off, r, D.pairs + P.pair_off, P.pair_cap);
    for (int k = threadIdx.x; k < min(n, min(cap, P.pair_cap)); k += kThreads) {
        int4 q = D.pairs[P.pair_off + k];
        out[3 * k] = q.x;
        out[3 * k + 1] = q.x == 0 ? D.vuser[M.xv_off + q.y] : q.y;   // gel vertex: input id
        out[3 * k + 2] = q.z;
    }
    if (threadIdx.x == 0) *count = n;
}

// marker readout: u_m = sum_k w_k u_{v_k}, first two components
__global__ void markers_kernel(const __grid_constant__ Dev D, float* out) {
    int pad = blockIdx.y;
    const PadDev P = D.pads[pad];
    const MeshDev M = D.meshes[P.mesh];
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M.n_mk) return;
    const int* id = D.mk_ids + kMarkerSlots * (M.mk_off + m);
    const float* w = D.mk_w + kMarkerSlots * (M.mk_off + m);
    for (int c = 0; c < 2; ++c) {
        float a = 0.f;
        for (int k = 0; k < kMarkerSlots; ++k) {
            int sc = c * D.Vt + P.v_off + id[k];
            a += w[k] * (D.uh[sc] + D.ul[sc]);
        }
        out[2 * (P.mk_out + m) + c] = a;
    }
}

// ---------------------------------------------------------------------------
// adjoint of a frame's equilibrium: H lambda = dL/dx by block-Jacobi PCG with
// a matrix-free Hessian-vector product, then dL/dtheta = -lambda^T dg/dtheta

// exact Hessian action of the barrier and lagged friction on the direction
// in p, written as slot values (3 force components, zero blocks)
// Hessian-vector product of the contact terms with p, into the slot buffer:
// the barrier part (when barrier is set) and the lagged friction part
__device__ __noinline__ void pair_hvp(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np, int nl,
                                      double s, bool barrier = true) {
    const int4* pr = D.pairs + P.pair_off;
    float* sb = D.slotbuf + (size_t)9 * 6 * P.pair_off;
    const double dh = P.dhat, kap = P.kappa;
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        float out[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        V3<float> Xf[4];
        load_slots<float>(D, P, M, gsl, isl, 0.0f, s, Xf);
        if (barrier && (double)pair_feature<float>(q.x, Xf).d <= 2.0 * dh) {
            V3<double> X[4], dl[4];
            load_slots<double>(D, P, M, gsl, isl, 0.0f, s, X);
            Feature<double> f = pair_feature<double>(q.x, X);
            if (f.d < dh && f.d > 0.0) {
#pragma unroll
                for (int sl = 0; sl < 4; ++sl) {
                    if (gsl[sl] >= 0) {
                        int si = P.v_off + gsl[sl];
                        dl[sl] = {D.p[si], D.p[D.Vt + si], D.p[2 * D.Vt + si]};
                    } else {
                        dl[sl] = {0.0, 0.0, 0.0};
                    }
                }
                double d1;
                V3<double> hv[4], rh;
                feat_hess_vec(f, X, dl, d1, hv, rh);
                const Barrier3 bb = barrier_all(f.d, dh);
                const EdgeMoll em = edge_moll(X, ee_eps(D, M, E, q.x, gsl, isl));
                double b1 = kap * em.m * bb.b1, b2 = kap * em.m * bb.b2;
                // mollified edge-edge terms: m'' c' b dc + m' b (Hess c) dl
                // + m' b' (d' dc + c' dd)
                double c1 = 0.0, c2 = 0.0;
                if (em.on) edge_moll_dir(em, dl, c1, c2);
#pragma unroll
                for (int sl = 0; sl < 3; ++sl)
                    if (gsl[sl] >= 0) {
                        double a = b2 * d1 * f.w[sl];
                        V3<double> o = a * rh + b1 * hv[sl];
                        if (em.on) {
                            const V3<double> gc = edge_moll_grad(em, sl);
                            o = o + (kap * (em.m2 * c1 * bb.b + em.m1 * bb.b1 * d1)) * gc +
                                (kap * em.m1 * bb.b) * edge_moll_hvec(em, dl, sl) +
                                (kap * em.m1 * c1 * bb.b1 * f.w[sl]) * rh;
                        }
                        out[sl][0] = (float)o.x;
                        out[sl][1] = (float)o.y;
                        out[sl][2] = (float)o.z;
                    }
            }
        }
#pragma unroll
        for (int sl = 0; sl < 3; ++sl)
            if (gsl[sl] >= 0) {
                float* e = sb + 9 * (3 * k + sl);
#pragma unroll
                for (int c = 0; c < 3; ++c) e[c] = out[sl][c];
#pragma unroll
                for (int c = 3; c < 9; ++c) e[c] = 0.f;
            }
    }
    const LagRec* lg = D.lag + P.pair_off;
    for (int l = threadIdx.x; l < nl; l += kThreads) {
        const LagRec& L = lg[l];
        double Dl[3] = {-s * L.dY[0], -s * L.dY[1], -s * L.dY[2]}, pd[3] = {0, 0, 0};
        for (int gs = 0; gs < 3; ++gs)
            if (L.g[gs] >= 0) {
                int si = P.v_off + L.g[gs];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    int sc = c * D.Vt + si;
                    Dl[c] += (double)L.w[gs] * (double)((D.uh[sc] - D.u0h[sc]) + (D.ul[sc] - D.u0l[sc]));
                    pd[c] += (double)L.w[gs] * (double)D.p[sc];
                }
            }
        double nD = L.n[0] * Dl[0] + L.n[1] * Dl[1] + L.n[2] * Dl[2];
        double tD[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) tD[c] = Dl[c] - L.n[c] * nD;
        double sv = sqrt(tD[0] * tD[0] + tD[1] * tD[1] + tD[2] * tD[2]);
        double eps = P.eps_v, cf = (double)P.mu_f * L.lam;
        double f1s = moll_f1_over_s(sv, eps), cs = moll_c(sv, eps);
        double uu[3] = {0, 0, 0};
        if (sv > 0)
#pragma unroll
            for (int c = 0; c < 3; ++c) uu[c] = tD[c] / sv;
        double npd = L.n[0] * pd[0] + L.n[1] * pd[1] + L.n[2] * pd[2];
        double upd = uu[0] * pd[0] + uu[1] * pd[1] + uu[2] * pd[2];
        double Hp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) Hp[c] = f1s * (pd[c] - L.n[c] * npd) - cs * uu[c] * upd;
        for (int gs = 0; gs < 3; ++gs)
            if (L.g[gs] >= 0) {
                float* e = sb + 9 * (3 * (P.pair_cap + l) + gs);
                double a = cf * L.w[gs];
#pragma unroll
                for (int c = 0; c < 3; ++c) e[c] = (float)(a * Hp[c]);
#pragma unroll
                for (int c = 3; c < 9; ++c) e[c] = 0.f;
            }
    }
    __syncthreads();
}

// dR(r)/dr_m of the rotation vector r (derivative of the Rodrigues formula)
__device__ void rotation_jacobian(const float* pose, double dR[3][9]) {
    double r[3] = {pose[0], pose[1], pose[2]};
    double th2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double R[9];
    rotation(pose, R);
    for (int m = 0; m < 3; ++m) {
        double K[9];
        if (th2 < 1e-16) {
            double e[3] = {0, 0, 0};
            e[m] = 1.0;
            double Km[9] = {0, -e[2], e[1], e[2], 0, -e[0], -e[1], e[0], 0};
            for (int q = 0; q < 9; ++q) dR[m][q] = Km[q];
            continue;
        }
        // v = r x ((I - R) e_m); K = (r_m [r]x + [v]x) / |r|^2; dR_m = K R
        double c[3] = {-R[m], -R[3 + m], -R[6 + m]};
        c[m] += 1.0;
        double v[3] = {r[1] * c[2] - r[2] * c[1], r[2] * c[0] - r[0] * c[2], r[0] * c[1] - r[1] * c[0]};
        double a[3] = {r[m] * r[0] + v[0], r[m] * r[1] + v[1], r[m] * r[2] + v[2]};
        double Kx[9] = {0, -a[2], a[1], a[2], 0, -a[0], -a[1], a[0], 0};
        for (int q = 0; q < 9; ++q) K[q] = Kx[q] / th2;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                dR[m][3 * i + j] = K[3 * i] * R[j] + K[3 * i + 1] * R[3 + j] + K[3 * i + 2] * R[6 + j];
    }
}

// lambda (in p) against dg/dtheta of the contact terms: out[0] the friction
// coefficient, out[1..6] the end pose (rotation vector, translation) through
// the mixed gel / indenter second derivatives, out[7..12] the start pose
// (dRs its rotation Jacobian), which enters only the lagged friction term,
// through the indenter's displacement over the frame
__device__ __noinline__ void pair_theta(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int np,
                                        int nl, const double dR[3][9], const double dRs[3][9], double out13[13]) {
    double acc[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const int4* pr = D.pairs + P.pair_off;
    const double dh = P.dhat, kap = P.kappa;
    auto dy_of = [&](int j, int m) -> V3<double> {
        if (m >= 3) {
            V3<double> e = {0, 0, 0};
            if (m == 3) e.x = 1.0;
            else if (m == 4) e.y = 1.0;
            else e.z = 1.0;
            return e;
        }
        const float* y = D.Y + 3 * (E.y_off + j);
        const double* A = dR[m];
        return V3<double>{A[0] * y[0] + A[1] * y[1] + A[2] * y[2], A[3] * y[0] + A[4] * y[1] + A[5] * y[2],
                          A[6] * y[0] + A[7] * y[1] + A[8] * y[2]};
    };
    auto dys_of = [&](int j, int m) -> V3<double> {
        if (m >= 3) return dy_of(j, m);
        const float* y = D.Y + 3 * (E.y_off + j);
        const double* A = dRs[m];
        return V3<double>{A[0] * y[0] + A[1] * y[1] + A[2] * y[2], A[3] * y[0] + A[4] * y[1] + A[5] * y[2],
                          A[6] * y[0] + A[7] * y[1] + A[8] * y[2]};
    };
    for (int k = threadIdx.x; k < np; k += kThreads) {
        int gsl[4], isl[4];
        int4 q = pr[k];
        pair_slots(D, M, E, q, gsl, isl);
        V3<float> Xf[4];
        load_slots<float>(D, P, M, gsl, isl, 0.0f, 1.0, Xf);
        if ((double)pair_feature<float>(q.x, Xf).d > 2.0 * dh) continue;
        V3<double> X[4];
        load_slots<double>(D, P, M, gsl, isl, 0.0f, 1.0, X);
        Feature<double> f = pair_feature<double>(q.x, X);
        if (!(f.d < dh && f.d > 0.0)) continue;
        const Barrier3 bb = barrier_all(f.d, dh);
        const EdgeMoll em = edge_moll(X, ee_eps(D, M, E, q.x, gsl, isl));
        V3<double> dl[4], dlam[4];
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            if (gsl[sl] >= 0) {
                int si = P.v_off + gsl[sl];
                dlam[sl] = {D.p[si], D.p[D.Vt + si], D.p[2 * D.Vt + si]};
            } else {
                dlam[sl] = {0.0, 0.0, 0.0};
            }
        }
        // mixed second derivatives by polarisation of the directional second
        // derivative Q(dl) of kappa m(c) b(d)
        double d1, d2;
        feat_dir_derivs(f, X, dlam, d1, d2);
        double Ql = kap * moll_barrier_dir2(em, dlam, d1, d2, bb);
        for (int m = 0; m < 6; ++m) {
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) dl[sl] = isl[sl] >= 0 ? dy_of(isl[sl], m) : V3<double>{0.0, 0.0, 0.0};
            feat_dir_derivs(f, X, dl, d1, d2);
            double Qd = kap * moll_barrier_dir2(em, dl, d1, d2, bb);
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) dl[sl] = dl[sl] + dlam[sl];
            feat_dir_derivs(f, X, dl, d1, d2);
            double Qs = kap * moll_barrier_dir2(em, dl, d1, d2, bb);
            acc[1 + m] += 0.5 * (Qs - Ql - Qd);
        }
    }
    const LagRec* lg = D.lag + P.pair_off;
    if (P.mu_f > 0.f)
        for (int l = threadIdx.x; l < nl; l += kThreads) {
            const LagRec& L = lg[l];
            double Dl[3] = {-L.dY[0], -L.dY[1], -L.dY[2]}, pd[3] = {0, 0, 0};
            for (int gs = 0; gs < 3; ++gs)
                if (L.g[gs] >= 0) {
                    int si = P.v_off + L.g[gs];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        int sc = c * D.Vt + si;
                        Dl[c] += (double)L.w[gs] * (double)((D.uh[sc] - D.u0h[sc]) + (D.ul[sc] - D.u0l[sc]));
                        pd[c] += (double)L.w[gs] * (double)D.p[sc];
                    }
                }
            double nD = L.n[0] * Dl[0] + L.n[1] * Dl[1] + L.n[2] * Dl[2];
            double tD[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) tD[c] = Dl[c] - L.n[c] * nD;
            double sv = sqrt(tD[0] * tD[0] + tD[1] * tD[1] + tD[2] * tD[2]);
            double eps = P.eps_v, cf = (double)P.mu_f * L.lam;
            double f1s = moll_f1_over_s(sv, eps), cs = moll_c(sv, eps);
            acc[0] += L.lam * f1s * (tD[0] * pd[0] + tD[1] * pd[1] + tD[2] * pd[2]);
            double uu[3] = {0, 0, 0};
            if (sv > 0)
#pragma unroll
                for (int c = 0; c < 3; ++c) uu[c] = tD[c] / sv;
            for (int m = 0; m < 6; ++m) {
                V3<double> dy = {0, 0, 0};
                for (int q = 0; q < 3; ++q)
                    if (L.iv[q] >= 0) dy = dy + (double)L.iw[q] * dy_of(L.iv[q], m);
                double a[3] = {dy.x, dy.y, dy.z};
                double na = L.n[0] * a[0] + L.n[1] * a[1] + L.n[2] * a[2];
                double ua = uu[0] * a[0] + uu[1] * a[1] + uu[2] * a[2];
                double Ha = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) Ha += pd[c] * (f1s * (a[c] - L.n[c] * na) - cs * uu[c] * ua);
                acc[1 + m] -= cf * Ha;
                // start pose: the displacement depends on -y^t, so the sign flips
                V3<double> ds = {0, 0, 0};
                for (int q = 0; q < 3; ++q)
                    if (L.iv[q] >= 0) ds = ds + (double)L.iw[q] * dys_of(L.iv[q], m);
                double b[3] = {ds.x, ds.y, ds.z};
                double nb = L.n[0] * b[0] + L.n[1] * b[1] + L.n[2] * b[2];
                double ub = uu[0] * b[0] + uu[1] * b[1] + uu[2] * b[2];
                double Hb = 0.0;
#pragma unroll
                for (int c = 0; c < 3; ++c) Hb += pd[c] * (f1s * (b[c] - L.n[c] * nb) - cs * uu[c] * ub);
                acc[7 + m] += cf * Hb;
            }
        }
    double first[8], rest[5];
#pragma unroll
    for (int q = 0; q < 8; ++q) first[q] = acc[q];
#pragma unroll
    for (int q = 0; q < 5; ++q) rest[q] = acc[8 + q];
    block_sum<8>(first);
    block_sum<5>(rest);
#pragma unroll
    for (int q = 0; q < 8; ++q) out13[q] = first[q];
#pragma unroll
    for (int q = 0; q < 5; ++q) out13[8 + q] = rest[q];
}

// z = P r with P the block-Jacobi inverse of (blk[gp] + m I); returns r.z, r.r
__device__ __noinline__ void pcg_precond(const Dev& D, const PadDev& P, const MeshDev& M, int gp, double& rz,
                                         double& rr) {
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
        if (D.fixed[M.xv_off + i]) {
#pragma unroll
            for (int c = 0; c < 3; ++c) D.z[c * D.Vt + si] = 0.f;
            continue;
        }
        float m = P.rho * D.vlump[M.xv_off + i];
        float K[6], Ki[6], r[3], z[3];
#pragma unroll
        for (int c = 0; c < 6; ++c) K[c] = D.blk[gp][c * D.Vt + si];
        K[0] += m; K[1] += m; K[2] += m;
        if (P.precond == 0) {
            if (!sym_inverse(K, Ki)) { Ki[0] = Ki[1] = Ki[2] = 1.f / m; Ki[3] = Ki[4] = Ki[5] = 0.f; }
        } else {
            Ki[0] = 1.f / K[0]; Ki[1] = 1.f / K[1]; Ki[2] = 1.f / K[2];
            Ki[3] = Ki[4] = Ki[5] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = D.adj_r[c * D.Vt + si];
        sym_apply(Ki, r, z);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            D.z[c * D.Vt + si] = z[c];
            v[0] += (double)r[c] * (double)z[c];
            v[1] += (double)r[c] * (double)r[c];
        }
    }
    block_sum<2>(v);
    rz = v[0];
    rr = v[1];
}

// q = H d: completes g[gq] (elastic + contact) with the mass term, zero on
// Dirichlet vertices; returns d . q
__device__ __noinline__ double hvp_finish(const Dev& D, const PadDev& P, const MeshDev& M, int gq) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
        bool fx = D.fixed[M.xv_off + i] != 0;
        float m = P.rho * D.vlump[M.xv_off + i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + si;
            float q = fx ? 0.f : D.g[gq][sc] + m * D.p[sc];
            D.g[gq][sc] = q;
            v[0] += (double)q * (double)D.p[sc];
        }
    }
    block_sum<1>(v);
    return v[0];
}

// x += alpha d, r -= alpha q (mode 0); d = z + beta d (mode 1); d = z (mode 2)
__device__ __noinline__ void pcg_vectors(const Dev& D, const PadDev& P, const MeshDev& M, int mode, double ab,
                                         int gq) {
    const float a = (float)ab;
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        int si = P.v_off + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int sc = c * D.Vt + si;
            if (mode == 0) {
                D.adj_x[sc] += a * D.p[sc];
                D.adj_r[sc] -= a * D.g[gq][sc];
            } else if (mode == 1) {
                D.p[sc] = D.z[sc] + a * D.p[sc];
            } else {
                D.p[sc] = D.z[sc];
            }
        }
    }
    __syncthreads();
}

// Installs a frame that was solved before, without solving it again, for the
// adjoint kernels: the start state (x0, v0; caller order [Vt][3]) with the
// start pose in pose_t, the end pose in pose_n, and the end positions x1.
// The friction lag is rebuilt from the start state and pose by the same
// steps as the solve's frame setup (broad phase at the start, lag_build), so
// that it equals the lag the frame was solved with when x0, v0 and the poses
// are the ones that solve started from.
__global__ void __launch_bounds__(kThreads) frame_install_kernel(const __grid_constant__ Dev D, const float* x0,
                                                                 const float* v0, const float* x1) {
    const int pad = blockIdx.x;
    load_pad(D, pad);
    const PadDev& P = S.P;
    const MeshDev& M = S.M;
    const EnvDev& E = S.E;
    world_indenter(D, P, E, D.pose_t + 6 * pad, D.Yt);
    world_indenter(D, P, E, D.pose_n + 6 * pad, D.Yn);
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        const size_t si = (size_t)P.v_off + i;
        const size_t u = (size_t)P.v_off + D.vuser[M.xv_off + i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t sc = c * (size_t)D.Vt + si;
            const float hi = x0[3 * u + c] - D.X[c * (size_t)D.XVt + M.xv_off + i];
            const float v = v0[3 * u + c];
            D.uh[sc] = hi;
            D.ul[sc] = 0.f;
            D.vel[sc] = v;
            D.u0h[sc] = hi;
            D.u0l[sc] = 0.f;
            D.uhat[sc] = hi + P.h * v;
        }
    }
    __syncthreads();
    const double rbp = (P.dhat + P.dhat) * (1.0 + 1e-6);
    SrcState src{&D, &P, &M, 0.0f};
    int n = bp_build(src, D, M, E, D.ilist + P.il_off, rbp, D.pairs + P.pair_off, P.pair_cap);
    int nlag = lag_build_p(D, P, M, E, min(n, P.pair_cap));
    if (threadIdx.x == 0) D.pad_nlag[pad] = nlag;
    __syncthreads();
    for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
        const size_t si = (size_t)P.v_off + i;
        const size_t u = (size_t)P.v_off + D.vuser[M.xv_off + i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t sc = c * (size_t)D.Vt + si;
            const float hi = x1[3 * u + c] - D.X[c * (size_t)D.XVt + M.xv_off + i];
            D.uh[sc] = hi;
            D.ul[sc] = 0.f;
            D.vel[sc] = (x1[3 * u + c] - x0[3 * u + c]) / P.h;
        }
    }
}

enum { ADJ_CONVERGED = 0, ADJ_MAXITER = 1, ADJ_BREAKDOWN = 2, ADJ_NONFINITE = 3 };

// The friction lag's own dependence on the frame start, for the exact
// multi-frame adjoint. For a lag record, psi = lambda^T g_D(x*; lag) with
// the lag (normal force -kappa b'(d), normal, gel and indenter closest-point
// weights) rebuilt in float64 from the frame-start positions of the pair's
// primitives; the start positions that enter the friction displacement
// explicitly stay fixed (their part is the H_D lambda term). Central
// differences of psi (1e-10 m in positions and translation, 1e-7 rad in
// rotation) give, per record, -dpsi/dx^t of its gel slots, added to the
// record's slot entries (contact_gather sums them per vertex), and, summed
// over records into dps, dpsi/d(start pose).
__device__ __noinline__ void lag_relag(const Dev& D, const PadDev& P, const MeshDev& M, const EnvDev& E, int nl,
                                       int pad, double dps[6]) {
    double acc[6] = {0, 0, 0, 0, 0, 0};
    float* sb = D.slotbuf + (size_t)9 * 6 * P.pair_off;
    const LagRec* lg = D.lag + P.pair_off;
    const double dh = P.dhat, kap = P.kappa, eps = P.eps_v, muf = P.mu_f;
    double pose_s[6], pose_n[6];
    for (int m = 0; m < 6; ++m) {
        pose_s[m] = D.pose_s[6 * pad + m];
        pose_n[m] = D.pose_t[6 * pad + m];
    }
    double Rs[9], Rn[9];
    rotation_dd(pose_s, Rs);
    rotation_dd(pose_n, Rn);
    auto world = [&](const double R[9], const double* pose, int j) {
        const float* y = D.Y + 3 * (E.y_off + j);
        return V3<double>{R[0] * y[0] + R[1] * y[1] + R[2] * y[2] + pose[3],
                          R[3] * y[0] + R[4] * y[1] + R[5] * y[2] + pose[4],
                          R[6] * y[0] + R[7] * y[1] + R[8] * y[2] + pose[5]};
    };
    for (int l = threadIdx.x; l < nl; l += kThreads) {
        const LagRec& L = lg[l];
        const int4 q = make_int4(L.pq[0], L.pq[1], L.pq[2], 0);
        int gsl[4], isl[4];
        pair_slots(D, M, E, q, gsl, isl);
        V3<double> X0[4], Xe[4], la[4];
        for (int sl = 0; sl < 4; ++sl) {
            la[sl] = {0.0, 0.0, 0.0};
            if (gsl[sl] >= 0) {
                const int xi = M.xv_off + gsl[sl], si = P.v_off + gsl[sl];
                double a0[3], a1[3];
                for (int c = 0; c < 3; ++c) {
                    const int sc = c * D.Vt + si;
                    const double Xr = D.X[c * D.XVt + xi];
                    a0[c] = Xr + ((double)D.u0h[sc] + (double)D.u0l[sc]);
                    a1[c] = Xr + ((double)D.uh[sc] + (double)D.ul[sc]);
                }
                X0[sl] = {a0[0], a0[1], a0[2]};
                Xe[sl] = {a1[0], a1[1], a1[2]};
                la[sl] = {D.adj_x[si], D.adj_x[D.Vt + si], D.adj_x[2 * D.Vt + si]};
            } else {
                X0[sl] = world(Rs, pose_s, isl[sl]);
                Xe[sl] = world(Rn, pose_n, isl[sl]);
            }
        }
        // psi at frame-start primitive positions Xp (X0, Xe fixed in the displacement)
        const double eps_x = ee_eps(D, M, E, q.x, gsl, isl);
        auto psi = [&](const V3<double> Xp[4]) -> double {
            Feature<double> f = pair_feature<double>(q.x, Xp);
            if (!(f.d > 0.0) || f.d >= dh) return 0.0;      // the lag force vanishes there
            V3<double> r = feat_r(f, Xp);
            const double inv = 1.0 / f.d;
            const V3<double> n = inv * r;
            const double lamn = -kap * edge_moll(Xp, eps_x).m * barrier_b1(f.d, dh);
            V3<double> Dl = {0.0, 0.0, 0.0}, lw = {0.0, 0.0, 0.0};
            for (int sl = 0; sl < 4; ++sl) {
                // gel slots carry w >= 0, indenter slots w <= 0: sum w (x_e - x_0) is
                // the gel closest point's displacement minus the indenter's
                const V3<double> dx = {Xe[sl].x - X0[sl].x, Xe[sl].y - X0[sl].y, Xe[sl].z - X0[sl].z};
                Dl = {Dl.x + f.w[sl] * dx.x, Dl.y + f.w[sl] * dx.y, Dl.z + f.w[sl] * dx.z};
                if (gsl[sl] >= 0) lw = {lw.x + f.w[sl] * la[sl].x, lw.y + f.w[sl] * la[sl].y, lw.z + f.w[sl] * la[sl].z};
            }
            const double nD = dot(n, Dl);
            const V3<double> t = {Dl.x - nD * n.x, Dl.y - nD * n.y, Dl.z - nD * n.z};
            const double sg = sqrt(dot(t, t));
            return muf * lamn * moll_f1_over_s(sg, eps) * dot(lw, t);
        };
        V3<double> Xp[4];
        for (int sl = 0; sl < 4; ++sl) Xp[sl] = X0[sl];
        const double hx = 1e-10;
        for (int sl = 0; sl < 3; ++sl) {
            if (gsl[sl] < 0) continue;
            float* e = sb + 9 * (3 * (P.pair_cap + l) + sl);
            for (int c = 0; c < 3; ++c) {
                double* xc = c == 0 ? &Xp[sl].x : (c == 1 ? &Xp[sl].y : &Xp[sl].z);
                const double x0 = *xc;
                *xc = x0 + hx;
                const double p1 = psi(Xp);
                *xc = x0 - hx;
                const double p2 = psi(Xp);
                *xc = x0;
                e[c] += (float)(-(p1 - p2) / (2.0 * hx));
            }
        }
        for (int m = 0; m < 6; ++m) {
            const double hm = m < 3 ? 1e-7 : 1e-10;
            double pv[2];
            for (int sg = 0; sg < 2; ++sg) {
                double pp[6];
                for (int k = 0; k < 6; ++k) pp[k] = pose_s[k];
                pp[m] += sg == 0 ? hm : -hm;
                double Rp[9];
                rotation_dd(pp, Rp);
                for (int sl = 0; sl < 4; ++sl) Xp[sl] = isl[sl] >= 0 ? world(Rp, pp, isl[sl]) : X0[sl];
                pv[sg] = psi(Xp);
            }
            acc[m] += (pv[0] - pv[1]) / (2.0 * hm);
        }
    }
    double v6[6] = {acc[0], acc[1], acc[2], acc[3], acc[4], acc[5]};
    block_sum<6>(v6);
    for (int m = 0; m < 6; ++m) dps[m] = v6[m];
}


// Adjoint of the last frame. dLdm (markers) and dLdx (caller-order end
// positions) form the right-hand side, either may be null. out: per pad
// out_stride doubles (9: Lame pair, mu_f, end pose; 15: plus the start pose).
// dx0 / dv0 (caller order, may be null): dL/dx^t = (M + H_D) lambda and
// dL/dv^t = h M lambda with the frame's friction lag held fixed (H_D the
// lagged friction Hessian).
__global__ void __launch_bounds__(kThreads, 2) adjoint_kernel(const __grid_constant__ Dev D, const float* dLdm,
                                                              const float* dLdx, double* out, int out_stride,
                                                              float* dx0, float* dv0, int* status, int* iters,
                                                              int max_iter, float tol, int relag) {
    const int pad = blockIdx.x;
    load_pad(D, pad);
    const PadDev& P = S.P;
    const MeshDev& M = S.M;
    const EnvDev& E = S.E;
    if (threadIdx.x == 0) S.flag = 0;
    __syncthreads();
    // candidates at the equilibrium with the indenter at the frame's end
    SrcState src{&D, &P, &M, 1.0f};
    int n = bp_build(src, D, M, E, D.ilist + P.il_off, (P.dhat + P.dhat) * (1.0 + 1e-6), D.pairs + P.pair_off,
                     P.pair_cap);
    ContactCtl cc{min(n, P.pair_cap), D.pad_nlag[pad], 0};
    csr_build(D, P, M, E, cc);
    // preconditioner blocks at x* (buffer 0)
    TetOut t0 = tet_pass<1>(D, P, M, 0.0f, 0);
    double rem;
    int bad;
    float fsc;
    pair_trial<double>(D, P, M, E, cc.npairs, cc.nlag, 1.0, 0.0f, rem, bad, fsc);
    contact_gather(D, P, cc, 0);
    // right-hand side dL/dx (transpose of the marker readout), lambda = 0
    for (int i = threadIdx.x; i < M.n_v; i += kThreads)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            D.adj_r[c * D.Vt + P.v_off + i] = 0.f;
            D.adj_x[c * D.Vt + P.v_off + i] = 0.f;
        }
    __syncthreads();
    if (dLdx) {
        for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
            if (D.fixed[M.xv_off + i]) continue;
            const size_t u = (size_t)P.v_off + D.vuser[M.xv_off + i];
#pragma unroll
            for (int c = 0; c < 3; ++c) D.adj_r[c * D.Vt + P.v_off + i] = dLdx[3 * u + c];
        }
        __syncthreads();
    }
    if (dLdm && threadIdx.x == 0)
        for (int m = 0; m < M.n_mk; ++m)
            for (int k = 0; k < kMarkerSlots; ++k) {
                int v = D.mk_ids[kMarkerSlots * (M.mk_off + m) + k];
                float w = D.mk_w[kMarkerSlots * (M.mk_off + m) + k];
                if (D.fixed[M.xv_off + v]) continue;
                for (int c = 0; c < 2; ++c)
                    D.adj_r[c * D.Vt + P.v_off + v] += w * dLdm[2 * (P.mk_out + m) + c];
            }
    __syncthreads();
    double rz, rr;
    pcg_precond(D, P, M, 0, rz, rr);
    const double bnorm = sqrt(rr);
    int st = (t0.bad || bad) ? ADJ_NONFINITE : ADJ_CONVERGED;
    int it = 0;
    if (st == ADJ_CONVERGED && bnorm > 0.0) {
        pcg_vectors(D, P, M, 2, 0.0, 1);
        st = ADJ_MAXITER;
        for (it = 0; it < max_iter; ++it) {
            tet_pass<2>(D, P, M, 0.0f, 1);
            pair_hvp(D, P, M, E, cc.npairs, cc.nlag, 1.0);
            contact_gather(D, P, cc, 1);
            double dq = hvp_finish(D, P, M, 1);
            if (!(dq > 0.0)) { st = ADJ_BREAKDOWN; break; }
            double alpha = rz / dq;
            pcg_vectors(D, P, M, 0, alpha, 1);
            double rz1;
            pcg_precond(D, P, M, 0, rz1, rr);
            if (!isfinite(rr)) { st = ADJ_NONFINITE; break; }
            if (sqrt(rr) <= (double)tol * bnorm) { st = ADJ_CONVERGED; ++it; break; }
            pcg_vectors(D, P, M, 1, rz1 / rz, 1);
            rz = rz1;
        }
    }
    // dL/dtheta = -lambda^T dg/dtheta
    for (int i = threadIdx.x; i < M.n_v; i += kThreads)
#pragma unroll
        for (int c = 0; c < 3; ++c) D.p[c * D.Vt + P.v_off + i] = D.adj_x[c * D.Vt + P.v_off + i];
    __syncthreads();
    TetOut t3 = tet_pass<3>(D, P, M, 0.0f, 0);
    double dR[3][9], dRs[3][9];
    rotation_jacobian(D.pose_t + 6 * pad, dR);
    rotation_jacobian(D.pose_s + 6 * pad, dRs);
    double c13[13];
    pair_theta(D, P, M, E, cc.npairs, cc.nlag, dR, dRs, c13);
    if (threadIdx.x == 0) {
        double* o = out + (size_t)out_stride * pad;
        o[0] = -t3.acc;
        o[1] = -t3.acc2;
        for (int q = 0; q < 7; ++q) o[2 + q] = -c13[q];
        if (out_stride >= 15)
            for (int q = 0; q < 6; ++q) o[9 + q] = -c13[7 + q];
        if (status) status[pad] = st;
        if (iters) iters[pad] = it;
    }
    if (dx0 || dv0 || relag) {
        // H_D lambda: the lagged friction part of the Hessian-vector product
        // (p holds lambda), gathered into g[1]; with relag the lag's own
        // dependence on the frame start joins the same slot entries
        for (int i = threadIdx.x; i < M.n_v; i += kThreads)
#pragma unroll
            for (int c = 0; c < 3; ++c) D.g[1][c * D.Vt + P.v_off + i] = 0.f;
        __syncthreads();
        pair_hvp(D, P, M, E, cc.npairs, cc.nlag, 1.0, false);
        if (relag && P.mu_f > 0.f) {
            double dps[6];
            lag_relag(D, P, M, E, cc.nlag, pad, dps);
            if (threadIdx.x == 0 && out_stride >= 15) {
                double* o = out + (size_t)out_stride * pad;
                for (int q = 0; q < 6; ++q) o[9 + q] -= dps[q];
            }
        }
        contact_gather(D, P, cc, 1);
        for (int i = threadIdx.x; i < M.n_v; i += kThreads) {
            const size_t si = (size_t)P.v_off + i;
            const size_t u = (size_t)P.v_off + D.vuser[M.xv_off + i];
            const bool fx = D.fixed[M.xv_off + i] != 0;
            const float m = P.rho * D.vlump[M.xv_off + i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float l = D.adj_x[c * D.Vt + si];
                if (dx0) dx0[3 * u + c] = fx ? 0.f : m * l + D.g[1][c * D.Vt + si];
                if (dv0) dv0[3 * u + c] = fx ? 0.f : P.h * m * l;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// allocation-free broad phase: the same candidate search as broadphase_kernel
// on caller arrays, with its scratch (culled indenter primitives and the
// staged candidate list) in one fixed array of this file instead of the
// batch's device memory.

constexpr int kStaticScratchInt4 = 1 << 16;        // 1 MiB per device
static __device__ __align__(256) int4 g_static_scratch[kStaticScratchInt4];

__global__ void __launch_bounds__(kThreads) broadphase_static_kernel2(const __grid_constant__ Dev D,
                                                                      const __grid_constant__ MeshDev M,
                                                                      const __grid_constant__ EnvDev E,
                                                                      const float* x, const float* y, double r,
                                                                      int4* scratch, int n_list_int4, int* out,
                                                                      int cap, int* count) {
    SrcArrays src{x, y, nullptr};
    int* ilist = reinterpret_cast<int*>(scratch);
    int4* staged = scratch + n_list_int4;
    int n = bp_build(src, D, M, E, ilist, r, staged, cap);
    for (int k = threadIdx.x; k < min(n, cap); k += kThreads) {
        int4 q = staged[k];
        out[3 * k] = q.x;
        out[3 * k + 1] = q.y;
        out[3 * k + 2] = q.z;
    }
    if (threadIdx.x == 0) *count = n;
}

#endif  // TAC_WIDE

// ---------------------------------------------------------------------------
// host side: dynamic shared memory of the kernels that use the CTA scratch

size_t shared_bytes() { return sizeof(Shared); }

#ifdef TAC_WIDE
cudaError_t configure_kernels() {
    return cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
}
}  // namespace wide
}  // namespace tac
#else
cudaError_t configure_kernels() {
    int bytes = (int)sizeof(Shared);
    cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(debug_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(frame_install_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(broadphase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace tac

// ---------------------------------------------------------------------------
// allocation-free entry point (declared in include/tac.h)

#include <mutex>
#include <string>

#include "tac.h"

namespace tac {
void set_last_error(const std::string& msg);   // message returned by tac_last_error (api.cu)
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};      // device address of g_static_scratch, per device

int static_fail(int code, const std::string& m) {
    tac::set_last_error(m);
    return code;
}

}  // namespace

extern "C" int tac_broadphase_static(const float* x_dev, const int* surf_verts_dev, int n_surf_verts,
                                     const int* surf_tris_dev, int n_surf_tris, const int* surf_edges_dev,
                                     int n_surf_edges, const float* y_dev, int n_ind_verts,
                                     const int* ind_tris_dev, int n_ind_tris, const int* ind_edges_dev,
                                     int n_ind_edges, double r, int* pairs_out_dev, int capacity, int* count_dev,
                                     void* stream) {
    using namespace tac;
    if (!x_dev || !y_dev || !pairs_out_dev || !count_dev || n_surf_verts < 0 || n_surf_tris < 0 ||
        n_surf_edges < 0 || n_ind_verts <= 0 || n_ind_tris < 0 || n_ind_edges < 0 || capacity < 0 || !(r >= 0) ||
        (n_surf_verts && !surf_verts_dev) || (n_surf_tris && !surf_tris_dev) || (n_surf_edges && !surf_edges_dev) ||
        (n_ind_tris && !ind_tris_dev) || (n_ind_edges && !ind_edges_dev))
        return static_fail(TAC_ERR_INVALID_ARG, "tac_broadphase_static: null pointer or negative size");
    // scratch: culled indenter primitive ids (rounded up to int4) + staged candidates
    long long n_list = (long long)n_ind_tris + n_ind_verts + n_ind_edges;
    long long n_list_int4 = (n_list + 3) / 4;
    if (n_list_int4 + capacity > kStaticScratchInt4)
        return static_fail(TAC_ERR_INVALID_ARG,
                           "tac_broadphase_static: indenter primitives + 4 x capacity exceed the fixed scratch of " +
                               std::to_string(4 * kStaticScratchInt4) + " ints (1 MiB)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return static_fail(TAC_ERR_CUDA, "tac_broadphase_static: no usable current device");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            // first call on this device: look up the device address of the
            // fixed array (the host-side symbol is only a stand-in for it)
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_static_scratch);
            if (e != cudaSuccess)
                return static_fail(TAC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            e = configure_kernels();
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(broadphase_static_kernel2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)shared_bytes());
            if (e != cudaSuccess)
                return static_fail(TAC_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
            g_static_ptr[dev] = ptr;
        }
        scratch = g_static_ptr[dev];
    }
    Dev D{};
    MeshDev M{};
    EnvDev E{};
    M.n_sv = n_surf_verts;
    M.n_st = n_surf_tris;
    M.n_se = n_surf_edges;
    E.n_v = n_ind_verts;
    E.n_t = n_ind_tris;
    E.n_e = n_ind_edges;
    D.sv = surf_verts_dev;
    D.st = surf_tris_dev;
    D.se = surf_edges_dev;
    D.it = ind_tris_dev;
    D.ie = ind_edges_dev;
    D.meshes = nullptr;
    D.envs = nullptr;
    broadphase_static_kernel2<<<1, kThreads, shared_bytes(), static_cast<cudaStream_t>(stream)>>>(
        D, M, E, x_dev, y_dev, r, static_cast<int4*>(scratch), (int)n_list_int4, pairs_out_dev, capacity, count_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(TAC_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return TAC_OK;
}
#endif  // TAC_WIDE
