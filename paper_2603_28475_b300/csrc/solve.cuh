// Device-side data of a batch and the per-pad PNCG-IPC frame solve.
//
// One CTA owns one pad for a whole frame: it moves the indenter along its
// path in CCD-bounded substeps, keeps the contact candidate set valid, and
// runs the preconditioned nonlinear CG (Supp. A, Eq. dk_direction and
// Eq. step_size) to convergence with only CTA-level barriers. The tet passes
// stream warp-sized spatial patches of <= 32 tets through per-warp shared
// memory stages; per-corner contributions are summed per vertex through the
// patch's corner CSR (a deterministic segmented reduction, no atomics), and
// patches of one colour class share no vertex.
#pragma once

#include <cstdint>

#include "device_math.cuh"
#include "layout.h"

namespace tac {

constexpr int kThreads = 256;
constexpr int kStage = 4 * kPatchTets;  // corner slots of one warp-sized tet patch

struct MeshDev {
    int xv_off, n_v;          // static per-vertex arrays (X, vlump, fixed)
    int tet_off, n_t;         // tet arrays (B, lconn, slot): kPatchTets slots per patch; n_t real tets
    int n_patch;              // patch q: tet slots tet_off + 32 q, vertex entries pvert_off + 32 q,
                              // CSR offsets pcsr_off + 33 q
    int col_off, n_col;       // colour classes: patches [colour[col_off+c], colour[col_off+c+1])
    int pvert_off, pcsr_off;
    int sv_off, n_sv, st_off, n_st, se_off, n_se;
    int mk_off, n_mk;
    int dm_off, n_dm;         // Dm^-1 table entries [dm_off, dm_off + n_dm) (n_dm = 0: per-tet B)
};

struct EnvDev {
    int y_off, n_v, t_off, n_t, e_off, n_e;
};

struct PadDev {
    int mesh, env;
    int v_off;                // state vertex offset
    int yw_off;               // per-pad world indenter vertex slots
    int pair_off, pair_cap;   // candidate pairs (and lag records, entries)
    int il_off;               // per-pad culled indenter primitive list
    int mk_out;               // marker output offset (markers)
    float mu, lam, rho, h, dhat, kappa, mu_f, eps_v, g_ref, tol, tol_adv;
    float floor;              // float32 resolution floor of the stopping target, per unit F_max
    int max_iter, precond;
    int step;                 // 0: alpha bounded by CCD + Armijo test; 1: Eq. (step_size) as printed
    int prec;                 // 0: float64 contact features, bounds and sums; 1: the plain-FP32 form
};

struct LagRec {
    int g[3];                 // gel vertex (mesh-local id) of each gel slot, -1 if none
    float w[3];               // gel slot weights
    float n[3];               // lagged contact normal
    float dY[3];              // indenter closest-point displacement over the frame
    int iv[3];                // indenter vertex (env-local id) of each indenter slot, -1 if none
    float iw[3];              // indenter slot weights (>= 0)
    double lam;               // lagged normal force magnitude -kappa b'(d)
    int pq[3];                // the candidate pair it was built from (type, i, j)
};

// All device arrays of a batch (SoA with strides noted).
struct Dev {
    int n_pads, Vt;           // pads, state vertices
    const MeshDev* meshes;
    const EnvDev* envs;
    const PadDev* pads;
    const int* order;         // pads in processing order
    // static mesh data
    const float* X;           // [3][XVt] rest positions
    int XVt;
    const float* vlump;       // [XVt]
    const float* wdiag;       // [XVt] static diagonal of the elastic blocks / (h^2 mu)
    const uint8_t* fixed;     // [XVt]
    const int* vuser;         // [XVt] internal vertex -> input vertex id (mesh-local)
    const float* B;           // [9][Tt], Tt = total tet slots (zero for meshes with a Dm^-1 table)
    const float* dm_table;    // [sum n_dm * 9] distinct Dm^-1 of tabled meshes
    int Tt;
    const uint32_t* lconn;    // [Tt]
    const uint32_t* slot;     // [Tt] 4 x 8-bit corner slots
    const int* colour;        // per mesh colour offsets into its patch list
    const int* pvert;
    const uint16_t* pcsr;
    const int* sv;
    const int* st;            // [n*3]
    const int* se;            // [n*2]
    const int* mk_ids;        // [n*kMarkerSlots]
    const float* mk_w;        // [n*kMarkerSlots]
    // indenters
    const float* Y;           // [n*3] local
    const int* it;            // [n*3]
    const int* ie;            // [n*2]
    float* Yt;                // [n*3] world at the frame start (per pad slots)
    float* Yn;                // [n*3] world at the frame end
    const float* pose_t;      // [n_pads*6]
    const float* pose_n;      // [n_pads*6]
    const float* pose_s;      // [n_pads*6] start pose of the last solved frame
    // state [c][Vt]
    float *uh, *ul, *u0h, *u0l, *vel, *uhat, *p, *z;
    float* g[2];              // [3][Vt]
    float* blk[2];            // [6][Vt]
    // contact scratch (per pad regions of pair_cap)
    int4* pairs;
    LagRec* lag;
    float* slotbuf;           // [6 * pair_cap][9] per pad region (pairs then lag, 3 slots each)
    double* bpair;            // [pair_cap] per pad: barrier value b(d) of each pair at the current point
    Feature<double>* fcache;  // [pair_cap] per pad: float64 feature of each pair at the last trial point
                              // (nf = -1: farther than the float64 band, d its float32 bound)
    int* ent;                 // [6 * pair_cap]
    int* cvl;                 // [6 * pair_cap + 1] contact vertex list / offsets
    int* cvo;                 // [6 * pair_cap + 1]
    int* cnt;                 // [Vt] zero between uses
    int* ilist;               // culled indenter primitives
    // outputs
    int* status;
    int* iters;
    long long* stats;         // [n_pads][16] counters and per-phase nanoseconds
    double* norms;            // [n_pads][4] final |g|_inf, stopping target, g_ref, force scale
    int* pad_nlag;            // [n_pads] lag records of the last frame
    float* adj_x;             // [3][Vt] adjoint solution lambda
    float* adj_r;             // [3][Vt] adjoint residual
    int* queue;
};

}  // namespace tac
