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

namespace tac {

constexpr int kPatchTets = 32;
constexpr int kPatchVerts = 32;
constexpr int kPatchCsr = kPatchVerts + 1;
constexpr uint32_t kNoTet = 0xffffffffu;

// Marker map: every marker reads kMarkerSlots weighted mesh vertices (a
// barycentric map fills three and gives the fourth weight 0).
constexpr int kMarkerSlots = 4;

// Flags carried in the high bits of a patch's vertex entry (entries >= 0).
constexpr int kFirstFlag = 1 << 30;   // first patch (in processing order) touching the vertex
constexpr int kLastFlag = 1 << 29;    // last patch touching the vertex
constexpr int kVertMask = (1 << 29) - 1;

}  // namespace tac
