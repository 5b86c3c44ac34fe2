// Layout constants of the tet patches, shared by the host preprocessing
// (mesh.cpp) and the device passes (kernels.cu).
//
// A patch is processed by one warp with one tet per lane and one vertex per
// lane when its corner contributions are reduced. Patches are stored with a
// fixed stride (kPatchTets tet slots, kPatchVerts vertex entries, kPatchCsr
// CSR offsets), so a patch's data is addressed from its index alone; unused
// tet slots carry kNoTet local ids, unused vertex entries -1 and empty CSR
// runs.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define TAC_HD __host__ __device__
#else
#define TAC_HD
#endif

namespace tac {

constexpr int kPatchTets = 32;
constexpr int kPatchVerts = 32;
constexpr int kPatchCsr = kPatchVerts + 1;
constexpr uint32_t kNoTet = 0xffffffffu;
// warps of one solve CTA: the scatter passes take a colour class's patches
// in rounds of kCtaWarps (one patch per warp)
constexpr int kCtaWarps = 8;

// Marker map: every marker reads kMarkerSlots weighted mesh vertices (a
// barycentric map fills three and gives the fourth weight 0).
constexpr int kMarkerSlots = 4;

// Rest-shape table: a mesh with at most kMaxDmTypes distinct Dm^-1 (a regular
// hex-split grid has 6, one per tet of the cell split) keeps them in a table
// and tags each tet with its table index in the spare high bits of its local
// vertex ids (3 bits of byte 0, 2 bits of byte 1; local ids take 5 bits).
constexpr int kMaxDmTypes = 32;
constexpr uint32_t kLocalMask = 31u;
TAC_HD inline uint32_t dm_type_bits(int t) {
    return (static_cast<uint32_t>(t & 7) << 5) | (static_cast<uint32_t>((t >> 3) & 3) << 13);
}
TAC_HD inline int dm_type_of(uint32_t lc) {
    return static_cast<int>(((lc >> 5) & 7u) | (((lc >> 13) & 3u) << 3));
}

// Flags carried in the high bits of a patch's vertex entry (entries >= 0).
constexpr int kFirstFlag = 1 << 30;   // first patch (in processing order) touching the vertex
constexpr int kLastFlag = 1 << 29;    // last patch touching the vertex
constexpr int kVertMask = (1 << 29) - 1;

}  // namespace tac
