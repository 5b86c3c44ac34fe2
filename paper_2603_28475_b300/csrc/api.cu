// Host implementation of the C ABI declared in include/tac.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "mesh.h"
#include "solve.cuh"
#include "tac.h"

namespace tac {
__global__ void solve_kernel(const __grid_constant__ Dev D);
__global__ void debug_eval_kernel(const __grid_constant__ Dev D, float alpha, double r, float* grad_out, float* blk_out, double* scal);
__global__ void broadphase_kernel(const __grid_constant__ Dev D, int pad, const float* x, const float* y, double r, int* out, int cap,
                                  int* count);
__global__ void markers_kernel(const __grid_constant__ Dev D, float* out);
__global__ void schedule_kernel(const __grid_constant__ Dev D, unsigned long long* key, int* idx, int n2, int* order);
__global__ void frame_install_kernel(const __grid_constant__ Dev D, const float* x0, const float* v0, const float* x1);
__global__ void adjoint_kernel(const __grid_constant__ Dev D, const float* dLdm, const float* dLdx, double* out,
                               int out_stride, float* dx0, float* dv0, int* status, int* iters, int max_iter, float tol,
                               int relag);
size_t shared_bytes();
cudaError_t configure_kernels();
void set_last_error(const std::string& msg);
namespace wide {   // the 512-thread block shape of the solve kernel (kernels_wide.cu)
constexpr int kThreads = 512;
__global__ void solve_kernel(const __grid_constant__ Dev D);
size_t shared_bytes();
cudaError_t configure_kernels();
}  // namespace wide
}  // namespace tac

using namespace tac;

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

}  // namespace

void tac::set_last_error(const std::string& msg) { g_err = msg; }

namespace {

#define CUDA_TRY(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(TAC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---- small helper kernels ---------------------------------------------------

// Caller arrays are [Vt][3] in input vertex order (pad by pad); the state is
// SoA in the internal vertex order. u2i maps a caller index to its state index.
__global__ void aos_to_state(const float* x, const float* X, int XVt, const int* xv_of_state, const int* u2i,
                             float* uh, float* ul, int Vt, bool subtract_rest) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vt) return;
    int j = u2i[i];
    int xi = xv_of_state[j];
    for (int c = 0; c < 3; ++c) {
        float v = x[3 * i + c];
        if (subtract_rest) v -= X[c * XVt + xi];
        uh[c * Vt + j] = v;
        if (ul) ul[c * Vt + j] = 0.f;
    }
}

__global__ void state_to_aos(const float* uh, const float* ul, const float* X, int XVt, const int* xv_of_state,
                             const int* u2i, float* out, int Vt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vt) return;
    int j = u2i[i];
    int xi = xv_of_state[j];
    for (int c = 0; c < 3; ++c) {
        float v = uh[c * Vt + j];
        if (ul) v += ul[c * Vt + j];
        if (X) v += X[c * XVt + xi];
        out[3 * i + c] = v;
    }
}

__global__ void copy_aos_to_soa(const float* a, const int* u2i, float* s, int Vt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Vt) return;
    int j = u2i[i];
    for (int c = 0; c < 3; ++c) s[c * Vt + j] = a[3 * i + c];
}

// target pose = current pose advanced by h * twist (rotation composed with
// exp(h w) on the left, translation += h v)
__global__ void integrate_twist(const float* pose_t, const float* twist, const float* hstep, float* pose_n, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* p = pose_t + 6 * i;
    const float* w = twist + 6 * i;
    double h = hstep[i];
    auto rot = [](const double r[3], double R[9]) {
        double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        double k[3] = {0, 0, 0}, sn = 0, c1 = 0;
        if (th > 1e-300) {
            k[0] = r[0] / th; k[1] = r[1] / th; k[2] = r[2] / th;
            sn = sin(th);
            c1 = 1.0 - cos(th);
        }
        double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double kk = 0;
                for (int q = 0; q < 3; ++q) kk += K[3 * a + q] * K[3 * q + b];
                R[3 * a + b] = (a == b) + sn * K[3 * a + b] + c1 * kk;
            }
    };
    double r0[3] = {p[0], p[1], p[2]}, dw[3] = {h * w[0], h * w[1], h * w[2]};
    double R0[9], Rw[9], R[9];
    rot(r0, R0);
    rot(dw, Rw);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0;
            for (int q = 0; q < 3; ++q) s += Rw[3 * a + q] * R0[3 * q + b];
            R[3 * a + b] = s;
        }
    // rotation vector of R (log map)
    double tr = R[0] + R[4] + R[8];
    double ct = fmin(1.0, fmax(-1.0, 0.5 * (tr - 1.0)));
    double th = acos(ct);
    double v[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
    double sc = th < 1e-8 ? 0.5 : th / (2.0 * sin(th));
    if (th > 3.14159) {  // near pi: axis from the symmetric part
        double a[3] = {sqrt(fmax(0.0, (R[0] + 1) / 2)), sqrt(fmax(0.0, (R[4] + 1) / 2)), sqrt(fmax(0.0, (R[8] + 1) / 2))};
        if (R[1] < 0) a[1] = -a[1];
        if (R[2] < 0) a[2] = -a[2];
        for (int c = 0; c < 3; ++c) pose_n[6 * i + c] = (float)(th * a[c]);
    } else {
        for (int c = 0; c < 3; ++c) pose_n[6 * i + c] = (float)(sc * v[c]);
    }
    for (int c = 0; c < 3; ++c) pose_n[6 * i + 3 + c] = (float)(p[3 + c] + h * w[3 + c]);
}

template <class T>
T* dalloc(std::vector<void*>& keep, size_t n, int& rc) {
    if (n == 0) n = 1;
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
        rc = TAC_ERR_OOM;
        return nullptr;
    }
    keep.push_back(p);
    return static_cast<T*>(p);
}

}  // namespace

struct tac_batch {
    int device = 0;
    int n_pads = 0, n_envs = 0, ppe = 1;
    int Vt = 0, XVt = 0, Tt = 0, total_markers = 0, pair_cap = 0;
    int grid = 0;                   // CTAs of a 256-thread solve launch
    int grid_wide = 0;              // CTAs of a 512-thread solve launch
    int shape = 256;                // block shape of tac_step's solve launch (tac_set_block_shape)
    std::vector<tac_params> params;
    std::vector<PadMesh> meshes;
    std::vector<IndenterMesh> inds;
    std::vector<int> pad_mesh, env_ind;
    std::vector<MeshDev> hmesh;
    std::vector<PadDev> hpad;
    std::vector<EnvDev> henv;
    std::vector<float> hstep;       // per pad h (for twists)
    std::vector<void*> allocs;
    Dev dev{};
    // device-only helpers
    MeshDev* d_meshes = nullptr;
    PadDev* d_pads = nullptr;
    EnvDev* d_envs = nullptr;
    int* d_xv_of_state = nullptr;
    int* d_u2i = nullptr;                   // caller vertex index -> state index
    float* d_hstep = nullptr;
    float* d_pose_t = nullptr;
    float* d_pose_s = nullptr;              // start pose of the last tac_step
    float* d_pose_n = nullptr;
    int* d_order = nullptr;                 // processing order, rewritten before each solve
    unsigned long long* d_sched_key = nullptr;
    int* d_sched_idx = nullptr;
    int sched_n2 = 1;                       // next power of two >= n_pads
};

namespace {

void fill_pad_params(tac_batch* b, int p) {
    const tac_params& q = b->params[p];
    PadDev& P = b->hpad[p];
    const PadMesh& M = b->meshes[b->pad_mesh[p]];
    P.mu = (float)(q.E / (2.0 * (1.0 + q.nu)));
    P.lam = (float)(q.E * q.nu / ((1.0 + q.nu) * (1.0 - 2.0 * q.nu)));
    P.rho = q.rho;
    P.h = q.h;
    P.dhat = q.dhat;
    P.kappa = q.kappa > 0 ? q.kappa : (float)((double)q.h * q.h * q.E * M.lbar);
    P.mu_f = q.mu_f;
    P.eps_v = q.eps_v > 0 ? q.eps_v : (float)(1e-3 * q.h);
    P.g_ref = (float)((double)q.h * q.h * q.E * M.lbar * q.dhat);
    P.tol = q.tol_rel_grad;
    P.tol_adv = q.tol_advance;
    P.max_iter = q.max_iter;
    P.precond = q.precond_mode;
    P.step = q.step_mode;
    P.prec = q.precision_mode;
    // a float32 gradient is resolved only down to a few hundred ulps of the
    // largest force component summed into it (elastic corner forces, barrier
    // and friction slot forces): floor_ulps * 2^-24 (256 by default)
    P.floor = (q.floor_ulps > 0.0f ? q.floor_ulps : 256.0f) / 16777216.0f;
    b->hstep[p] = q.h;
}

bool params_ok(const tac_params& q) {
    return q.E > 0 && q.nu > -1 && q.nu < 0.5f && q.rho > 0 && q.h > 0 && q.dhat > 0 && q.mu_f >= 0 &&
           q.tol_rel_grad > 0 && q.tol_advance > 0 && q.max_iter >= 0 && (q.precond_mode == 0 || q.precond_mode == 1) &&
           (q.step_mode == 0 || q.step_mode == 1) && (q.marker_mode == 0 || q.marker_mode == 1) &&
           (q.precision_mode == 0 || q.precision_mode == 1) && q.floor_ulps >= 0.0f;
}

}  // namespace

extern "C" {

const char* tac_last_error(void) { return g_err.c_str(); }

int tac_create_batch(const tac_pad_desc* pads, const tac_params* params, int n_pads, const tac_indenter_desc* indenters,
                     int n_envs, int pads_per_env, const tac_options* opts, void* stream, tac_handle* out) {
    if (!out) return fail(TAC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!pads || !params || !indenters || n_pads <= 0 || n_envs <= 0 || pads_per_env <= 0 ||
        n_pads > (1 << 24) || (long long)n_envs * pads_per_env != n_pads)
        return fail(TAC_ERR_INVALID_ARG, "need 0 < n_pads = n_envs * pads_per_env <= 2^24 and non-null arrays");
    for (int p = 0; p < n_pads; ++p)
        if (!params_ok(params[p])) return fail(TAC_ERR_INVALID_ARG, "invalid parameters for pad " + std::to_string(p));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    tac_batch* b = new tac_batch();
    b->n_pads = n_pads;
    b->n_envs = n_envs;
    b->ppe = pads_per_env;
    b->params.assign(params, params + n_pads);
    b->hstep.assign(n_pads, 0.f);
    int cap = (opts && opts->pair_capacity > 0) ? opts->pair_capacity : 16384;
    bool share = !opts || opts->share_meshes != 0;
    bool dm_tab = !opts || opts->no_dm_table == 0;
    b->pair_cap = cap;
    cudaGetDevice(&b->device);
    // host meshes (dedup by identical host arrays when sharing)
    std::map<std::vector<const void*>, int> seen;
    std::string err;
    for (int p = 0; p < n_pads; ++p) {
        const tac_pad_desc& d = pads[p];
        std::vector<const void*> key = {d.rest_xyz, d.tets, d.fixed_idx, d.marker_xy,
                                        (const void*)(intptr_t)d.n_verts, (const void*)(intptr_t)d.n_tets,
                                        (const void*)(intptr_t)d.n_fixed, (const void*)(intptr_t)d.n_markers,
                                        (const void*)(intptr_t)params[p].marker_mode};
        auto it = share ? seen.find(key) : seen.end();
        if (it != seen.end()) {
            b->pad_mesh.push_back(it->second);
            continue;
        }
        PadMesh M;
        if (!build_pad_mesh(d.n_verts, d.n_tets, d.n_fixed, d.n_markers, d.rest_xyz, d.tets, d.fixed_idx,
                            d.marker_xy, params[p].marker_mode, M, err)) {
            delete b;
            return fail(TAC_ERR_INVALID_MESH, "pad " + std::to_string(p) + ": " + err);
        }
        if (dm_tab) build_dm_table(M);
        int id = (int)b->meshes.size();
        b->meshes.push_back(std::move(M));
        b->pad_mesh.push_back(id);
        if (share) seen[key] = id;
    }
    std::map<std::vector<const void*>, int> iseen;
    for (int e = 0; e < n_envs; ++e) {
        const tac_indenter_desc& d = indenters[e];
        std::vector<const void*> key = {d.verts, d.tris, (const void*)(intptr_t)d.n_verts,
                                        (const void*)(intptr_t)d.n_tris};
        auto it = iseen.find(key);
        if (it != iseen.end()) {
            b->env_ind.push_back(it->second);
            continue;
        }
        IndenterMesh I;
        if (!build_indenter_mesh(d.n_verts, d.n_tris, d.verts, d.tris, I, err)) {
            delete b;
            return fail(TAC_ERR_INVALID_MESH, "indenter " + std::to_string(e) + ": " + err);
        }
        int id = (int)b->inds.size();
        b->inds.push_back(std::move(I));
        b->env_ind.push_back(id);
        iseen[key] = id;
    }
    // layouts
    int XVt = 0, Tt = 0, pv_tot = 0, pc_tot = 0, sv_tot = 0, st_tot = 0, se_tot = 0, mk_tot = 0;
    int col_tot = 0, dm_tot = 0;
    for (auto& M : b->meshes) {
        MeshDev md{};
        md.xv_off = XVt; md.n_v = M.n_v;
        md.tet_off = Tt; md.n_t = M.n_t;
        md.n_patch = M.n_patch();
        md.pvert_off = pv_tot; md.pcsr_off = pc_tot;
        md.sv_off = sv_tot; md.n_sv = (int)M.sv.size();
        md.st_off = st_tot; md.n_st = (int)(M.st.size() / 3);
        md.se_off = se_tot; md.n_se = (int)(M.se.size() / 2);
        md.mk_off = mk_tot; md.n_mk = M.n_mk;
        md.col_off = col_tot; md.n_col = M.n_colour();
        md.dm_off = dm_tot; md.n_dm = M.n_dm_types();
        dm_tot += md.n_dm;
        col_tot += (int)M.colour_off.size();
        XVt += M.n_v; Tt += M.n_slots(); pv_tot += (int)M.pvert.size();
        pc_tot += (int)M.pcsr.size(); sv_tot += md.n_sv; st_tot += md.n_st; se_tot += md.n_se; mk_tot += M.n_mk;
        b->hmesh.push_back(md);
    }
    int y_tot = 0, t_tot = 0, e_tot = 0;
    for (auto& I : b->inds) {
        EnvDev ed{y_tot, I.n_v, t_tot, I.n_t, e_tot, I.n_e};
        y_tot += I.n_v; t_tot += I.n_t; e_tot += I.n_e;
        b->henv.push_back(ed);
    }
    int Vt = 0, yw = 0, il = 0, mko = 0;
    b->hpad.resize(n_pads);
    std::vector<int> xv_of_state;
    int vt_all = 0;
    for (int p = 0; p < n_pads; ++p) vt_all += b->hmesh[b->pad_mesh[p]].n_v;
    std::vector<int> u2i(vt_all);
    for (int p = 0; p < n_pads; ++p) {
        PadDev& P = b->hpad[p];
        const MeshDev& md = b->hmesh[b->pad_mesh[p]];
        const EnvDev& ed = b->henv[b->env_ind[p / pads_per_env]];
        P.mesh = b->pad_mesh[p];
        P.env = b->env_ind[p / pads_per_env];
        P.v_off = Vt;
        P.yw_off = yw;
        P.pair_off = p * cap;
        P.pair_cap = cap;
        P.il_off = il;
        P.mk_out = mko;
        for (int i = 0; i < md.n_v; ++i) xv_of_state.push_back(md.xv_off + i);
        const PadMesh& pm = b->meshes[P.mesh];
        for (int i = 0; i < md.n_v; ++i) u2i[Vt + pm.vuser[i]] = Vt + i;
        Vt += md.n_v;
        yw += ed.n_v;
        il += ed.n_t + ed.n_v + ed.n_e;
        mko += md.n_mk;
        fill_pad_params(b, p);
    }
    b->Vt = Vt;
    b->XVt = XVt;
    b->Tt = Tt;
    b->total_markers = mko;
    // processing order: larger meshes first (longest jobs start first)
    std::vector<int> order(n_pads);
    for (int p = 0; p < n_pads; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return b->hmesh[b->hpad[a].mesh].n_t > b->hmesh[b->hpad[c].mesh].n_t;
    });
    // device allocations
    int rc = TAC_OK;
    auto& K = b->allocs;
    Dev& D = b->dev;
    D.n_pads = n_pads;
    D.Vt = Vt;
    D.XVt = XVt;
    D.Tt = Tt;
    float* X = dalloc<float>(K, 3 * (size_t)XVt, rc);
    float* vlump = dalloc<float>(K, XVt, rc);
    float* wdiag = dalloc<float>(K, XVt, rc);
    uint8_t* fixed = dalloc<uint8_t>(K, XVt, rc);
    float* B = dalloc<float>(K, 9 * (size_t)Tt, rc);
    float* dm_table = dalloc<float>(K, 9 * (size_t)dm_tot, rc);
    uint32_t* lconn = dalloc<uint32_t>(K, Tt, rc);
    uint32_t* slot = dalloc<uint32_t>(K, Tt, rc);
    int* pvert = dalloc<int>(K, pv_tot, rc);
    uint16_t* pcsr = dalloc<uint16_t>(K, pc_tot, rc);
    int* sv = dalloc<int>(K, sv_tot, rc);
    int* stt = dalloc<int>(K, 3 * (size_t)st_tot, rc);
    int* se = dalloc<int>(K, 2 * (size_t)se_tot, rc);
    int* mk_ids = dalloc<int>(K, kMarkerSlots * (size_t)mk_tot, rc);
    float* mk_w = dalloc<float>(K, kMarkerSlots * (size_t)mk_tot, rc);
    float* Y = dalloc<float>(K, 3 * (size_t)y_tot, rc);
    int* it = dalloc<int>(K, 3 * (size_t)t_tot, rc);
    int* ie = dalloc<int>(K, 2 * (size_t)e_tot, rc);
    float* Yt = dalloc<float>(K, 3 * (size_t)yw, rc);
    float* Yn = dalloc<float>(K, 3 * (size_t)yw, rc);
    b->d_pose_t = dalloc<float>(K, 6 * (size_t)n_pads, rc);
    b->d_pose_s = dalloc<float>(K, 6 * (size_t)n_pads, rc);
    b->d_pose_n = dalloc<float>(K, 6 * (size_t)n_pads, rc);
    float* st3[8];
    for (int k = 0; k < 8; ++k) st3[k] = dalloc<float>(K, 3 * (size_t)Vt, rc);
    float* g0 = dalloc<float>(K, 3 * (size_t)Vt, rc);
    float* g1 = dalloc<float>(K, 3 * (size_t)Vt, rc);
    float* k0 = dalloc<float>(K, 6 * (size_t)Vt, rc);
    float* k1 = dalloc<float>(K, 6 * (size_t)Vt, rc);
    size_t pc = (size_t)n_pads * cap;
    int4* pairs = dalloc<int4>(K, pc, rc);
    LagRec* lag = dalloc<LagRec>(K, pc, rc);
    float* slotbuf = dalloc<float>(K, 9 * 6 * pc, rc);
    double* bpair = dalloc<double>(K, pc, rc);
    Feature<double>* fcache = dalloc<Feature<double>>(K, pc, rc);
    int* ent = dalloc<int>(K, 6 * pc, rc);
    int* cvl = dalloc<int>(K, 6 * pc + 1, rc);
    int* cvo = dalloc<int>(K, 6 * pc + 1, rc);
    int* cnt = dalloc<int>(K, Vt, rc);
    int* ilist = dalloc<int>(K, il, rc);
    int* colour = dalloc<int>(K, col_tot, rc);
    long long* stats = dalloc<long long>(K, 16 * (size_t)n_pads, rc);
    double* norms = dalloc<double>(K, 4 * (size_t)n_pads, rc);
    int* pad_nlag = dalloc<int>(K, n_pads, rc);
    float* adj_x = dalloc<float>(K, 3 * (size_t)Vt, rc);
    float* adj_r = dalloc<float>(K, 3 * (size_t)Vt, rc);
    int* queue = dalloc<int>(K, 1, rc);
    int* order_d = dalloc<int>(K, n_pads, rc);
    b->d_order = order_d;
    while (b->sched_n2 < n_pads) b->sched_n2 <<= 1;
    b->d_sched_key = dalloc<unsigned long long>(K, b->sched_n2, rc);
    b->d_sched_idx = dalloc<int>(K, b->sched_n2, rc);
    b->d_meshes = dalloc<MeshDev>(K, b->hmesh.size(), rc);
    b->d_pads = dalloc<PadDev>(K, n_pads, rc);
    b->d_envs = dalloc<EnvDev>(K, b->henv.size(), rc);
    b->d_xv_of_state = dalloc<int>(K, Vt, rc);
    b->d_u2i = dalloc<int>(K, Vt, rc);
    int* vuser = dalloc<int>(K, XVt, rc);
    b->d_hstep = dalloc<float>(K, n_pads, rc);
    if (rc != TAC_OK) {
        tac_destroy_batch(b);
        return fail(TAC_ERR_OOM, "device allocation failed");
    }
    // host staging of static data
    std::vector<float> hwd(XVt);
    std::vector<float> hX(3 * (size_t)XVt), hvl(XVt), hB(9 * (size_t)Tt), hmkw, hY;
    std::vector<uint8_t> hfx(XVt);
    std::vector<int> hvu(XVt);
    std::vector<uint32_t> hlc(Tt);
    std::vector<uint32_t> hsl(Tt);
    std::vector<int> hcol;
    std::vector<int> hpv, hsv, hst, hse, hmki, hit, hie;
    std::vector<uint16_t> hpc;
    std::vector<float> hdm;
    for (size_t m = 0; m < b->meshes.size(); ++m) {
        const PadMesh& M = b->meshes[m];
        const MeshDev& md = b->hmesh[m];
        for (int i = 0; i < M.n_v; ++i) {
            for (int c = 0; c < 3; ++c) hX[(size_t)c * XVt + md.xv_off + i] = M.X[3 * i + c];
            hvl[md.xv_off + i] = M.vlump[i];
            hwd[md.xv_off + i] = M.wdiag[i];
            hfx[md.xv_off + i] = M.fixed[i];
            hvu[md.xv_off + i] = M.vuser[i];
        }
        const int ns = M.n_slots();
        // a tabled mesh's per-tet Dm^-1 stays zero on the device: nothing reads it
        const bool tabled = md.n_dm > 0;
        hdm.insert(hdm.end(), M.dm_table.begin(), M.dm_table.end());
        for (int t = 0; t < ns; ++t) {
            if (!tabled)
                for (int e = 0; e < 9; ++e) hB[(size_t)e * Tt + md.tet_off + t] = M.B[(size_t)e * ns + t];
            hlc[md.tet_off + t] = M.lconn[t];
            hsl[md.tet_off + t] = M.slot[t];
        }
        hpv.insert(hpv.end(), M.pvert.begin(), M.pvert.end());
        hpc.insert(hpc.end(), M.pcsr.begin(), M.pcsr.end());
        hsv.insert(hsv.end(), M.sv.begin(), M.sv.end());
        hst.insert(hst.end(), M.st.begin(), M.st.end());
        hse.insert(hse.end(), M.se.begin(), M.se.end());
        hmki.insert(hmki.end(), M.mk_ids.begin(), M.mk_ids.end());
        hmkw.insert(hmkw.end(), M.mk_w.begin(), M.mk_w.end());
        hcol.insert(hcol.end(), M.colour_off.begin(), M.colour_off.end());
    }
    for (auto& I : b->inds) {
        hY.insert(hY.end(), I.Y.begin(), I.Y.end());
        hit.insert(hit.end(), I.tris.begin(), I.tris.end());
        hie.insert(hie.end(), I.edges.begin(), I.edges.end());
    }
    auto up = [&](void* dst, const void* src, size_t bytes) -> int {
        if (bytes == 0) return TAC_OK;
        CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
        return TAC_OK;
    };
    int r2 = TAC_OK;
    r2 |= up(X, hX.data(), hX.size() * 4);
    r2 |= up(vlump, hvl.data(), hvl.size() * 4);
    r2 |= up(fixed, hfx.data(), hfx.size());
    r2 |= up(B, hB.data(), hB.size() * 4);
    r2 |= up(dm_table, hdm.data(), hdm.size() * 4);
    r2 |= up(lconn, hlc.data(), hlc.size() * 4);
    r2 |= up(slot, hsl.data(), hsl.size() * 4);
    r2 |= up(colour, hcol.data(), hcol.size() * 4);
    r2 |= up(pvert, hpv.data(), hpv.size() * 4);
    r2 |= up(pcsr, hpc.data(), hpc.size() * 2);
    r2 |= up(sv, hsv.data(), hsv.size() * 4);
    r2 |= up(stt, hst.data(), hst.size() * 4);
    r2 |= up(se, hse.data(), hse.size() * 4);
    r2 |= up(mk_ids, hmki.data(), hmki.size() * 4);
    r2 |= up(mk_w, hmkw.data(), hmkw.size() * 4);
    r2 |= up(Y, hY.data(), hY.size() * 4);
    r2 |= up(it, hit.data(), hit.size() * 4);
    r2 |= up(ie, hie.data(), hie.size() * 4);
    r2 |= up(b->d_meshes, b->hmesh.data(), b->hmesh.size() * sizeof(MeshDev));
    r2 |= up(b->d_pads, b->hpad.data(), b->hpad.size() * sizeof(PadDev));
    r2 |= up(b->d_envs, b->henv.data(), b->henv.size() * sizeof(EnvDev));
    r2 |= up(b->d_xv_of_state, xv_of_state.data(), xv_of_state.size() * 4);
    r2 |= up(b->d_u2i, u2i.data(), u2i.size() * 4);
    r2 |= up(wdiag, hwd.data(), hwd.size() * 4);
    r2 |= up(vuser, hvu.data(), hvu.size() * 4);
    r2 |= up(b->d_hstep, b->hstep.data(), b->hstep.size() * 4);
    r2 |= up(order_d, order.data(), order.size() * 4);
    if (r2 != TAC_OK) {
        std::string m = g_err;
        tac_destroy_batch(b);
        return fail(TAC_ERR_CUDA, m);
    }
    for (int k = 0; k < 8; ++k) CUDA_TRY(cudaMemsetAsync(st3[k], 0, 3 * (size_t)Vt * 4, st));
    CUDA_TRY(cudaMemsetAsync(g0, 0, 3 * (size_t)Vt * 4, st));
    CUDA_TRY(cudaMemsetAsync(g1, 0, 3 * (size_t)Vt * 4, st));
    CUDA_TRY(cudaMemsetAsync(k0, 0, 6 * (size_t)Vt * 4, st));
    CUDA_TRY(cudaMemsetAsync(k1, 0, 6 * (size_t)Vt * 4, st));
    CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)Vt * 4, st));
    CUDA_TRY(cudaMemsetAsync(stats, 0, 16 * (size_t)n_pads * 8, st));
    CUDA_TRY(cudaMemsetAsync(norms, 0, 4 * (size_t)n_pads * 8, st));
    CUDA_TRY(cudaMemsetAsync(pad_nlag, 0, (size_t)n_pads * 4, st));
    CUDA_TRY(cudaMemsetAsync(b->d_pose_t, 0, 6 * (size_t)n_pads * 4, st));
    CUDA_TRY(cudaMemsetAsync(b->d_pose_s, 0, 6 * (size_t)n_pads * 4, st));
    CUDA_TRY(cudaMemsetAsync(b->d_pose_n, 0, 6 * (size_t)n_pads * 4, st));
    D.meshes = b->d_meshes;
    D.envs = b->d_envs;
    D.pads = b->d_pads;
    D.order = order_d;
    D.X = X; D.vlump = vlump; D.wdiag = wdiag; D.fixed = fixed; D.vuser = vuser; D.B = B; D.dm_table = dm_table; D.lconn = lconn; D.slot = slot; D.colour = colour;
    D.pvert = pvert; D.pcsr = pcsr; D.sv = sv; D.st = stt; D.se = se;
    D.mk_ids = mk_ids; D.mk_w = mk_w; D.Y = Y; D.it = it; D.ie = ie; D.Yt = Yt; D.Yn = Yn;
    D.pose_t = b->d_pose_t; D.pose_n = b->d_pose_n; D.pose_s = b->d_pose_s;
    D.uh = st3[0]; D.ul = st3[1]; D.u0h = st3[2]; D.u0l = st3[3]; D.vel = st3[4]; D.uhat = st3[5];
    D.p = st3[6]; D.z = st3[7];
    D.g[0] = g0; D.g[1] = g1; D.blk[0] = k0; D.blk[1] = k1;
    D.pairs = pairs; D.lag = lag; D.slotbuf = slotbuf; D.bpair = bpair; D.fcache = fcache; D.ent = ent; D.cvl = cvl; D.cvo = cvo; D.cnt = cnt;
    D.ilist = ilist; D.stats = stats; D.norms = norms; D.queue = queue;
    D.pad_nlag = pad_nlag; D.adj_x = adj_x; D.adj_r = adj_r;
    D.status = nullptr; D.iters = nullptr;
    int nsm = 0, occ = 0;
    CUDA_TRY(configure_kernels());
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_kernel, kThreads, shared_bytes()));
    b->grid = std::max(1, std::min(n_pads, nsm * std::max(1, occ)));
    CUDA_TRY(wide::configure_kernels());
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wide::solve_kernel, wide::kThreads, wide::shared_bytes()));
    b->grid_wide = std::max(1, std::min(n_pads, nsm * std::max(1, occ)));
    CUDA_TRY(cudaStreamSynchronize(st));
    *out = b;
    return TAC_OK;
}

int tac_destroy_batch(tac_handle h) {
    if (!h) return fail(TAC_ERR_INVALID_ARG, "null handle");
    cudaDeviceSynchronize();
    for (void* p : h->allocs) cudaFree(p);
    delete h;
    return TAC_OK;
}

int tac_reset(tac_handle h, const float* pose6_dev, void* stream) {
    if (!h || !pose6_dev) return fail(TAC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t n3 = 3 * (size_t)h->Vt * 4;
    CUDA_TRY(cudaMemsetAsync(h->dev.uh, 0, n3, st));
    CUDA_TRY(cudaMemsetAsync(h->dev.ul, 0, n3, st));
    CUDA_TRY(cudaMemsetAsync(h->dev.vel, 0, n3, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_t, pose6_dev, 6 * (size_t)h->n_pads * 4, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_n, pose6_dev, 6 * (size_t)h->n_pads * 4, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_s, pose6_dev, 6 * (size_t)h->n_pads * 4, cudaMemcpyDeviceToDevice, st));
    return TAC_OK;
}

int tac_set_indenter(tac_handle h, const float* pose6_dev, const float* twist6_dev, void* stream) {
    if (!h || (!pose6_dev && !twist6_dev)) return fail(TAC_ERR_INVALID_ARG, "need a pose or a twist");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (pose6_dev) {
        CUDA_TRY(cudaMemcpyAsync(h->d_pose_n, pose6_dev, 6 * (size_t)h->n_pads * 4, cudaMemcpyDeviceToDevice, st));
    } else {
        integrate_twist<<<(h->n_pads + 127) / 128, 128, 0, st>>>(h->d_pose_t, twist6_dev, h->d_hstep, h->d_pose_n,
                                                                  h->n_pads);
        CUDA_TRY(cudaGetLastError());
    }
    return TAC_OK;
}

int tac_step(tac_handle h, int* pad_status_dev, int* iters_dev, void* stream) {
    if (!h) return fail(TAC_ERR_INVALID_ARG, "null handle");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Dev D = h->dev;
    D.status = pad_status_dev;
    D.iters = iters_dev;
    CUDA_TRY(cudaMemsetAsync(D.queue, 0, sizeof(int), st));
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_s, h->d_pose_t, 6 * (size_t)h->n_pads * 4, cudaMemcpyDeviceToDevice, st));
    // longest predicted pad first (its previous solve time, then its size)
    schedule_kernel<<<1, 1024, 0, st>>>(D, h->d_sched_key, h->d_sched_idx, h->sched_n2, h->d_order);
    CUDA_TRY(cudaGetLastError());
    if (h->shape == wide::kThreads)
        wide::solve_kernel<<<h->grid_wide, wide::kThreads, wide::shared_bytes(), st>>>(D);
    else
        solve_kernel<<<h->grid, kThreads, shared_bytes(), st>>>(D);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_t, h->d_pose_n, 6 * (size_t)h->n_pads * 4, cudaMemcpyDeviceToDevice, st));
    return TAC_OK;
}

int tac_markers(tac_handle h, float* out_dev, void* stream) {
    if (!h || !out_dev) return fail(TAC_ERR_INVALID_ARG, "null argument");
    int mx = 0;
    for (auto& m : h->hmesh) mx = std::max(mx, m.n_mk);
    if (mx == 0) return TAC_OK;
    dim3 grid((mx + 127) / 128, h->n_pads);
    markers_kernel<<<grid, 128, 0, static_cast<cudaStream_t>(stream)>>>(h->dev, out_dev);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_get_state(tac_handle h, float* x_dev, float* v_dev, void* stream) {
    if (!h) return fail(TAC_ERR_INVALID_ARG, "null handle");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int nb = (h->Vt + 255) / 256;
    if (x_dev) state_to_aos<<<nb, 256, 0, st>>>(h->dev.uh, h->dev.ul, h->dev.X, h->XVt, h->d_xv_of_state, h->d_u2i, x_dev, h->Vt);
    if (v_dev) state_to_aos<<<nb, 256, 0, st>>>(h->dev.vel, nullptr, nullptr, h->XVt, h->d_xv_of_state, h->d_u2i, v_dev, h->Vt);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_set_state(tac_handle h, const float* x_dev, const float* v_dev, void* stream) {
    if (!h || !x_dev || !v_dev) return fail(TAC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int nb = (h->Vt + 255) / 256;
    aos_to_state<<<nb, 256, 0, st>>>(x_dev, h->dev.X, h->XVt, h->d_xv_of_state, h->d_u2i, h->dev.uh, h->dev.ul, h->Vt, true);
    aos_to_state<<<nb, 256, 0, st>>>(v_dev, h->dev.X, h->XVt, h->d_xv_of_state, h->d_u2i, h->dev.vel, nullptr, h->Vt, false);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_set_params(tac_handle h, const tac_params* per_pad, int n) {
    if (!h || !per_pad || n != h->n_pads) return fail(TAC_ERR_INVALID_ARG, "need n_pads parameter sets");
    for (int p = 0; p < n; ++p)
        if (!params_ok(per_pad[p])) return fail(TAC_ERR_INVALID_ARG, "invalid parameters for pad " + std::to_string(p));
    for (int p = 0; p < n; ++p)
        if (per_pad[p].marker_mode != h->params[p].marker_mode)
            return fail(TAC_ERR_INVALID_ARG, "marker_mode is fixed at creation (pad " + std::to_string(p) + ")");
    h->params.assign(per_pad, per_pad + n);
    for (int p = 0; p < n; ++p) fill_pad_params(h, p);
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(h->d_pads, h->hpad.data(), h->hpad.size() * sizeof(PadDev), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h->d_hstep, h->hstep.data(), h->hstep.size() * 4, cudaMemcpyHostToDevice));
    return TAC_OK;
}

int tac_get_params(tac_handle h, tac_params* per_pad, int n) {
    if (!h || !per_pad || n != h->n_pads) return fail(TAC_ERR_INVALID_ARG, "need n_pads parameter slots");
    for (int p = 0; p < n; ++p) {
        per_pad[p] = h->params[p];
        per_pad[p].kappa = h->hpad[p].kappa;
        per_pad[p].eps_v = h->hpad[p].eps_v;
    }
    return TAC_OK;
}

int tac_broadphase(tac_handle h, int pad, const float* x_dev, const float* y_dev, double r, int* pairs_out_dev,
                   int capacity, int* count_dev, void* stream) {
    if (!h || pad < 0 || pad >= h->n_pads || !x_dev || !y_dev || !pairs_out_dev || !count_dev || capacity < 0 ||
        !(r >= 0))
        return fail(TAC_ERR_INVALID_ARG, "invalid argument");
    broadphase_kernel<<<1, kThreads, shared_bytes(), static_cast<cudaStream_t>(stream)>>>(h->dev, pad, x_dev, y_dev, r,
                                                                             pairs_out_dev, capacity, count_dev);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_debug_eval(tac_handle h, const float* u_dev, const float* p_dev, float alpha, float* grad_dev, float* blk_dev,
                   double* scal_dev, void* stream) {
    if (!h || !u_dev || !p_dev) return fail(TAC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int nb = (h->Vt + 255) / 256;
    aos_to_state<<<nb, 256, 0, st>>>(u_dev, h->dev.X, h->XVt, h->d_xv_of_state, h->d_u2i, h->dev.uh, h->dev.ul, h->Vt, false);
    copy_aos_to_soa<<<nb, 256, 0, st>>>(p_dev, h->d_u2i, h->dev.p, h->Vt);
    CUDA_TRY(cudaMemsetAsync(h->dev.vel, 0, 3 * (size_t)h->Vt * 4, st));
    double r = 2.0 * (double)h->hpad[0].dhat;
    debug_eval_kernel<<<h->n_pads, kThreads, shared_bytes(), st>>>(h->dev, alpha, r, grad_dev, blk_dev, scal_dev);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_stats(tac_handle h, long long* stats_dev, void* stream) {
    if (!h || !stats_dev) return fail(TAC_ERR_INVALID_ARG, "null argument");
    CUDA_TRY(cudaMemcpyAsync(stats_dev, h->dev.stats, 16 * (size_t)h->n_pads * 8, cudaMemcpyDeviceToDevice,
                             static_cast<cudaStream_t>(stream)));
    return TAC_OK;
}

int tac_adjoint(tac_handle h, const float* dL_dmarkers_dev, double* dL_dtheta_dev, int* status_dev, int* iters_dev,
                int max_iter, float tol, void* stream) {
    if (!h || !dL_dmarkers_dev || !dL_dtheta_dev || max_iter < 0 || !(tol > 0))
        return fail(TAC_ERR_INVALID_ARG, "invalid argument");
    adjoint_kernel<<<h->n_pads, kThreads, shared_bytes(), static_cast<cudaStream_t>(stream)>>>(
        h->dev, dL_dmarkers_dev, nullptr, dL_dtheta_dev, 9, nullptr, nullptr, status_dev, iters_dev, max_iter, tol, 0);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_set_frame(tac_handle h, const float* x0_dev, const float* v0_dev, const float* pose_start_dev,
                  const float* x1_dev, const float* pose_end_dev, void* stream) {
    if (!h || !x0_dev || !v0_dev || !pose_start_dev || !x1_dev || !pose_end_dev)
        return fail(TAC_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t pb = 6 * (size_t)h->n_pads * 4;
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_t, pose_start_dev, pb, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_n, pose_end_dev, pb, cudaMemcpyDeviceToDevice, st));
    frame_install_kernel<<<h->n_pads, kThreads, shared_bytes(), st>>>(h->dev, x0_dev, v0_dev, x1_dev);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_s, pose_start_dev, pb, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_pose_t, pose_end_dev, pb, cudaMemcpyDeviceToDevice, st));
    return TAC_OK;
}

int tac_adjoint_frame(tac_handle h, const float* dL_dmarkers_dev, const float* dL_dx_dev, double* dL_dtheta_dev,
                      float* dL_dx0_dev, float* dL_dv0_dev, int* status_dev, int* iters_dev, int max_iter, float tol,
                      int lag_mode, void* stream) {
    if (!h || !dL_dtheta_dev || max_iter < 0 || !(tol > 0) || (lag_mode != 0 && lag_mode != 1))
        return fail(TAC_ERR_INVALID_ARG, "invalid argument");
    adjoint_kernel<<<h->n_pads, kThreads, shared_bytes(), static_cast<cudaStream_t>(stream)>>>(
        h->dev, dL_dmarkers_dev, dL_dx_dev, dL_dtheta_dev, 15, dL_dx0_dev, dL_dv0_dev, status_dev, iters_dev,
        max_iter, tol, lag_mode);
    CUDA_TRY(cudaGetLastError());
    return TAC_OK;
}

int tac_pad_norms(tac_handle h, double* norms_dev, void* stream) {
    if (!h || !norms_dev) return fail(TAC_ERR_INVALID_ARG, "null argument");
    CUDA_TRY(cudaMemcpyAsync(norms_dev, h->dev.norms, 4 * (size_t)h->n_pads * 8, cudaMemcpyDeviceToDevice,
                             static_cast<cudaStream_t>(stream)));
    return TAC_OK;
}

int tac_marker_map(const tac_pad_desc* pad, int marker_mode, int* ids_host, float* w_host) {
    if (!pad || !ids_host || !w_host) return fail(TAC_ERR_INVALID_ARG, "null argument");
    if (marker_mode != 0 && marker_mode != 1) return fail(TAC_ERR_INVALID_ARG, "unknown marker mode");
    PadMesh M;
    std::string err;
    if (!build_pad_mesh(pad->n_verts, pad->n_tets, pad->n_fixed, pad->n_markers, pad->rest_xyz, pad->tets,
                        pad->fixed_idx, pad->marker_xy, marker_mode, M, err))
        return fail(TAC_ERR_INVALID_MESH, err);
    // the mesh stores internal vertex ids; report input ids
    for (size_t k = 0; k < M.mk_ids.size(); ++k) {
        ids_host[k] = M.vuser[M.mk_ids[k]];
        w_host[k] = M.mk_w[k];
    }
    return TAC_OK;
}

int tac_mesh_info(const tac_pad_desc* pad, int* n_patches, int* n_colours, int* n_dm_types, double* dm_dev,
                  int* n_rounds, int* n_conflicts) {
    if (!pad) return fail(TAC_ERR_INVALID_ARG, "null argument");
    PadMesh M;
    std::string err;
    if (!build_pad_mesh(pad->n_verts, pad->n_tets, pad->n_fixed, pad->n_markers, pad->rest_xyz, pad->tets,
                        pad->fixed_idx, pad->marker_xy, 0, M, err))
        return fail(TAC_ERR_INVALID_MESH, err);
    build_dm_table(M);
    if (n_patches) *n_patches = M.n_patch();
    if (n_colours) *n_colours = M.n_colour();
    if (n_dm_types) *n_dm_types = M.n_dm_types();
    if (dm_dev) *dm_dev = M.dm_dev;
    // scatter rounds (kCtaWarps patches each) and vertices shared within a class
    int rounds = 0, conflicts = 0;
    std::vector<int> seen(M.n_v, -1);
    for (int c = 0; c < M.n_colour(); ++c) {
        const int a = M.colour_off[c], e = M.colour_off[c + 1];
        rounds += (e - a + kCtaWarps - 1) / kCtaWarps;
        for (int q = a; q < e; ++q)
            for (int l = 0; l < kPatchVerts; ++l) {
                const int v = M.pvert[(size_t)q * kPatchVerts + l];
                if (v < 0) continue;
                const int id = v & kVertMask;
                if (seen[id] == c) ++conflicts;
                seen[id] = c;
            }
    }
    if (n_rounds) *n_rounds = rounds;
    if (n_conflicts) *n_conflicts = conflicts;
    return TAC_OK;
}

int tac_sizes(tac_handle h, int* total_verts, int* total_markers, int* pair_capacity, int* grid_ctas) {
    if (!h) return fail(TAC_ERR_INVALID_ARG, "null handle");
    if (total_verts) *total_verts = h->Vt;
    if (total_markers) *total_markers = h->total_markers;
    if (pair_capacity) *pair_capacity = h->pair_cap;
    if (grid_ctas) *grid_ctas = h->shape == wide::kThreads ? h->grid_wide : h->grid;
    return TAC_OK;
}

int tac_set_block_shape(tac_handle h, int threads) {
    if (!h) return fail(TAC_ERR_INVALID_ARG, "null handle");
    if (threads != kThreads && threads != wide::kThreads)
        return fail(TAC_ERR_INVALID_ARG, "block shape must be 256 or 512 threads");
    h->shape = threads;
    return TAC_OK;
}

int tac_autotune_block_shape(tac_handle h, const float* pose6_dev, int reps, int* threads_out, float* ms_out,
                             void* stream) {
    if (!h || !pose6_dev || !threads_out || reps < 1) return fail(TAC_ERR_INVALID_ARG, "null argument or reps < 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t n3 = 3 * (size_t)h->Vt, np = (size_t)h->n_pads;
    // the state a solve reads and writes: displacement (hi, lo), velocity,
    // the three pose arrays and the per-pad records the schedule keys on
    float* sv = nullptr;
    float* sp = nullptr;
    long long* ss = nullptr;
    int* si = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TAC_OK;
    auto release = [&]() {
        if (sv) cudaFree(sv);
        if (sp) cudaFree(sp);
        if (ss) cudaFree(ss);
        if (si) cudaFree(si);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    auto check = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == TAC_OK) rc = fail(TAC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    float* const state[3] = {h->dev.uh, h->dev.ul, h->dev.vel};
    float* const poses[3] = {h->d_pose_t, h->d_pose_n, h->d_pose_s};
    auto copy_state = [&](bool save) {
        for (int k = 0; k < 3; ++k) {
            float* a = sv + k * n3;
            check(cudaMemcpyAsync(save ? a : state[k], save ? state[k] : a, n3 * 4, cudaMemcpyDeviceToDevice, st),
                  "state copy");
            float* b = sp + k * 6 * np;
            check(cudaMemcpyAsync(save ? b : poses[k], save ? poses[k] : b, 6 * np * 4, cudaMemcpyDeviceToDevice, st),
                  "pose copy");
        }
        check(cudaMemcpyAsync(save ? ss : h->dev.stats, save ? h->dev.stats : ss, 16 * np * 8,
                              cudaMemcpyDeviceToDevice, st), "record copy");
    };
    if (check(cudaMalloc(&sv, 3 * n3 * 4), "cudaMalloc") && check(cudaMalloc(&sp, 18 * np * 4), "cudaMalloc") &&
        check(cudaMalloc(&ss, 16 * np * 8), "cudaMalloc") && check(cudaMalloc(&si, 2 * np * 4), "cudaMalloc") &&
        check(cudaEventCreate(&e0), "cudaEventCreate") && check(cudaEventCreate(&e1), "cudaEventCreate")) {
        copy_state(true);
        const int shapes[2] = {kThreads, wide::kThreads};
        float ms[2] = {0.f, 0.f};
        const int keep = h->shape;
        for (int c = 0; c < 2 && rc == TAC_OK; ++c) {
            h->shape = shapes[c];
            for (int r = 0; r < reps && rc == TAC_OK; ++r) {
                copy_state(false);
                int e = tac_set_indenter(h, pose6_dev, nullptr, stream);
                if (e == TAC_OK) check(cudaEventRecord(e0, st), "cudaEventRecord");
                if (e == TAC_OK) e = tac_step(h, si, si + np, stream);
                if (e != TAC_OK) {
                    rc = e;
                    break;
                }
                float t = 0.f;
                if (check(cudaEventRecord(e1, st), "cudaEventRecord") && check(cudaEventSynchronize(e1), "sync") &&
                    check(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime"))
                    ms[c] += t / (float)reps;
            }
        }
        copy_state(false);
        check(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        h->shape = keep;
        if (rc == TAC_OK) {
            h->shape = ms[1] < ms[0] ? wide::kThreads : kThreads;
            *threads_out = h->shape;
            if (ms_out) {
                ms_out[0] = ms[0];
                ms_out[1] = ms[1];
            }
        }
    }
    release();
    return rc;
}

}  // extern "C"
