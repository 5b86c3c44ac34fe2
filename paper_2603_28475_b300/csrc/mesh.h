// Host-side preprocessing of one gel pad mesh and one indenter mesh.
//
// Everything here runs once per distinct mesh at batch creation: validation,
// rest shape (Dm^-1 and lumped volume), canonical surface primitives, marker
// barycentric weights, and the spatial tet patches that the device kernels
// stream through shared memory.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "layout.h"

namespace tac {

struct PadMesh {
    int n_v = 0, n_t = 0, n_mk = 0;
    // Vertices are stored in an internal order (Morton order of the rest
    // positions); every vertex id below is internal unless noted.
    std::vector<int> vuser;           // [n_v] internal id -> input vertex id
    std::vector<float> X;             // [n_v*3] rest positions
    std::vector<float> vlump;         // [n_v] lumped rest volume (sum of V/4); mass = rho * vlump
    std::vector<float> wdiag;         // [n_v] sum over the vertex's corners of V |b|^2 (b: the corner's
                                      // row of the shape matrix); the elastic block's static diagonal
                                      // is h^2 mu wdiag
    std::vector<uint8_t> fixed;       // [n_v] 1 = Dirichlet
    // tets in patch order, kPatchTets slots per patch
    std::vector<float> B;             // [9][n_slots] Dm^-1 (row-major entries), SoA
    std::vector<float> dm_table;      // [n_types*9] rest-shape classes when there are at most
                                      // kMaxDmTypes (then lconn carries each tet's class); empty otherwise
    double dm_dev = 0.0;              // largest entry deviation of a tet from its class (relative)
    std::vector<uint32_t> lconn;      // [n_slots] 4 x 8-bit local vertex ids (kNoTet: unused slot)
    std::vector<uint32_t> slot;       // [n_slots] 4 x 8-bit corner slots in the patch CSR
    std::vector<int> patch;           // [n_patch*4] tet_begin, vert_begin, n_t | n_v << 16, csr_begin (host)
    std::vector<int> pvert;           // [n_patch*kPatchVerts] mesh vertex id | flags, -1 unused
    std::vector<uint16_t> pcsr;       // [n_patch*kPatchCsr] per patch CSR offsets
    std::vector<int> tet_order;       // slot -> input tet id (-1 unused)
    std::vector<int> colour_off;      // patches of colour c: [colour_off[c], colour_off[c+1])
    // canonical surface
    std::vector<int> sv;              // surface vertex ids, in increasing input id
    std::vector<int> st;              // [n_st*3] surface triangles, canonical order of the input ids
    std::vector<int> se;              // [n_se*2] surface edges, canonical order of the input ids
    double lbar = 0.0;                // mean rest surface edge length
    // markers
    std::vector<int> mk_ids;          // [n_mk*kMarkerSlots]
    std::vector<float> mk_w;          // [n_mk*kMarkerSlots]
    int n_dm_types() const { return static_cast<int>(dm_table.size() / 9); }
    int n_patch() const { return static_cast<int>(patch.size() / 4); }
    int n_slots() const { return n_patch() * kPatchTets; }
    int n_colour() const { return static_cast<int>(colour_off.size()) - 1; }
};

struct IndenterMesh {
    int n_v = 0, n_t = 0, n_e = 0;
    std::vector<float> Y;             // [n_v*3] local frame
    std::vector<int> tris;            // [n_t*3]
    std::vector<int> edges;           // [n_e*2] distinct (lo, hi), sorted
};

// Builds a pad; returns false with a message on invalid input. marker_mode
// selects the marker map (0 barycentric on the top face, 1 kNN inverse
// distance over the top-face nodes).
bool build_pad_mesh(int n_verts, int n_tets, int n_fixed, int n_markers, const float* rest,
                    const int* tets, const int* fixed, const float* markers, int marker_mode,
                    PadMesh& out, std::string& err);

// Groups the tet slots into rest-shape classes: Dm^-1 that agree entry by
// entry within kDmTableTol of the class representative's largest entry (a
// regular grid whose float32 coordinates differ from exact multiples of the
// cell size by rounding gives one class per tet of the cell split). With at
// most kMaxDmTypes classes, fills dm_table with the representatives, tags
// every slot's lconn with its class and returns true; otherwise leaves the
// mesh unchanged and returns false. The kernels form F = I + Du Dm^-1 from
// displacements, so a class representative perturbs the strain of a
// deformed tet by at most that relative amount and leaves the rest state
// exact.
constexpr double kDmTableTol = 1e-5;
bool build_dm_table(PadMesh& M);

// The marker map alone, in input vertex ids: ids/w [n_markers*kMarkerSlots].
// surf: canonical surface triangles (input ids), used by the barycentric map.
bool build_marker_map(int n_verts, const float* rest, const std::vector<int>& surf, int n_markers,
                      const float* markers, int marker_mode, std::vector<int>& ids, std::vector<float>& w,
                      std::string& err);

bool build_indenter_mesh(int n_verts, int n_tris, const float* verts, const int* tris,
                         IndenterMesh& out, std::string& err);

}  // namespace tac
