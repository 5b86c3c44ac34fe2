// Host-side mesh preprocessing (see mesh.h).
#include "mesh.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

namespace tac {

namespace {

uint32_t spread10(uint32_t v) {
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000ff;
    v = (v | (v << 8)) & 0x0300f00f;
    v = (v | (v << 4)) & 0x030c30c3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
}

double det3(const double m[9]) {
    return m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
           m[2] * (m[3] * m[7] - m[4] * m[6]);
}

void inv3(const double m[9], double o[9]) {
    double d = det3(m);
    o[0] = (m[4] * m[8] - m[5] * m[7]) / d;
    o[1] = (m[2] * m[7] - m[1] * m[8]) / d;
    o[2] = (m[1] * m[5] - m[2] * m[4]) / d;
    o[3] = (m[5] * m[6] - m[3] * m[8]) / d;
    o[4] = (m[0] * m[8] - m[2] * m[6]) / d;
    o[5] = (m[2] * m[3] - m[0] * m[5]) / d;
    o[6] = (m[3] * m[7] - m[4] * m[6]) / d;
    o[7] = (m[1] * m[6] - m[0] * m[7]) / d;
    o[8] = (m[0] * m[4] - m[1] * m[3]) / d;
}

char msgbuf[256];

}  // namespace

bool build_marker_map(int nv, const float* rest, const std::vector<int>& surf, int nm, const float* markers,
                      int mode, std::vector<int>& ids, std::vector<float>& w, std::string& err) {
    if (mode != 0 && mode != 1) {
        err = "unknown marker mode";
        return false;
    }
    ids.assign(kMarkerSlots * static_cast<size_t>(nm), 0);
    w.assign(kMarkerSlots * static_cast<size_t>(nm), 0.0f);
    if (nm == 0) return true;
    float ztop = rest[2];
    for (int i = 0; i < nv; ++i) ztop = std::max(ztop, rest[3 * i + 2]);
    if (mode == 0) {
        // the top-face triangle maximising the marker's smallest barycentric
        // coordinate (the containing triangle; first in canonical order on a tie)
        std::vector<int> top;
        const size_t nst = surf.size() / 3;
        for (size_t k = 0; k < nst; ++k) {
            const int* f = &surf[3 * k];
            if (rest[3 * f[0] + 2] == ztop && rest[3 * f[1] + 2] == ztop && rest[3 * f[2] + 2] == ztop)
                top.push_back(static_cast<int>(k));
        }
        for (int m = 0; m < nm; ++m) {
            double qx = markers[2 * m], qy = markers[2 * m + 1];
            double best = -1e300, bw[3] = {0, 0, 0};
            int bk = -1;
            for (int k : top) {
                const int* f = &surf[3 * static_cast<size_t>(k)];
                double ax = rest[3 * f[0]], ay = rest[3 * f[0] + 1];
                double v0x = rest[3 * f[1]] - ax, v0y = rest[3 * f[1] + 1] - ay;
                double v1x = rest[3 * f[2]] - ax, v1y = rest[3 * f[2] + 1] - ay;
                double v2x = qx - ax, v2y = qy - ay;
                double den = v0x * v1y - v1x * v0y;
                double l1 = (v2x * v1y - v1x * v2y) / den;
                double l2 = (v0x * v2y - v2x * v0y) / den;
                double l0 = 1.0 - l1 - l2;
                double sc = std::min(l0, std::min(l1, l2));
                if (sc > best) {
                    best = sc;
                    bk = k;
                    bw[0] = l0;
                    bw[1] = l1;
                    bw[2] = l2;
                }
            }
            if (bk < 0 || best < -1e-9) {
                std::snprintf(msgbuf, sizeof msgbuf, "marker %d is not on the top face", m);
                err = msgbuf;
                return false;
            }
            for (int r = 0; r < 3; ++r) {
                ids[kMarkerSlots * m + r] = surf[3 * static_cast<size_t>(bk) + r];
                w[kMarkerSlots * m + r] = static_cast<float>(bw[r]);
            }
            ids[kMarkerSlots * m + 3] = ids[kMarkerSlots * m];   // weight 0
        }
        return true;
    }
    // kNN inverse distance (Sec. 3.2): the kMarkerSlots top-face nodes nearest
    // to the marker in the face's 2-D distance, ranked by (dx^2 + dy^2, id);
    // weights 1/d normalised in rank order; a node at distance 0 takes all
    std::vector<int> top;
    for (int i = 0; i < nv; ++i)
        if (rest[3 * i + 2] == ztop) top.push_back(i);
    if (static_cast<int>(top.size()) < kMarkerSlots) {
        err = "fewer top-face nodes than marker neighbours";
        return false;
    }
    std::vector<std::pair<double, int>> key(top.size());
    for (int m = 0; m < nm; ++m) {
        double qx = markers[2 * m], qy = markers[2 * m + 1];
        for (size_t k = 0; k < top.size(); ++k) {
            int i = top[k];
            double dx = static_cast<double>(rest[3 * i]) - qx, dy = static_cast<double>(rest[3 * i + 1]) - qy;
            key[k] = {dx * dx + dy * dy, i};
        }
        std::partial_sort(key.begin(), key.begin() + kMarkerSlots, key.end());
        double inv[kMarkerSlots], sum = 0.0;
        bool on_node = key[0].first == 0.0;
        for (int r = 0; r < kMarkerSlots; ++r) {
            ids[kMarkerSlots * m + r] = key[r].second;
            inv[r] = on_node ? 0.0 : 1.0 / std::sqrt(key[r].first);
            sum += inv[r];
        }
        for (int r = 0; r < kMarkerSlots; ++r)
            w[kMarkerSlots * m + r] = on_node ? (r == 0 ? 1.0f : 0.0f) : static_cast<float>(inv[r] / sum);
    }
    return true;
}

bool build_dm_table(PadMesh& M) {
    // greedy classes in slot order: a tet joins the first class whose
    // representative (its first member's Dm^-1) agrees with its own entry by
    // entry within kDmTableTol of the representative's largest entry
    const size_t ns = static_cast<size_t>(M.n_slots());
    std::vector<std::array<float, 9>> rep;
    std::vector<float> rep_scale;
    std::vector<int> tag(ns, -1);
    double dev = 0.0;
    for (size_t t = 0; t < ns; ++t) {
        if (M.lconn[t] == kNoTet) continue;
        std::array<float, 9> b;
        for (int e = 0; e < 9; ++e) b[e] = M.B[e * ns + t];
        int found = -1;
        double fdev = 0.0;
        for (size_t k = 0; k < rep.size() && found < 0; ++k) {
            double worst = 0.0;
            for (int e = 0; e < 9; ++e) worst = std::max(worst, std::fabs(static_cast<double>(b[e]) - rep[k][e]));
            if (worst <= kDmTableTol * rep_scale[k]) {
                found = static_cast<int>(k);
                fdev = worst / rep_scale[k];
            }
        }
        if (found < 0) {
            if (static_cast<int>(rep.size()) == kMaxDmTypes) return false;
            float sc = 0.f;
            for (int e = 0; e < 9; ++e) sc = std::max(sc, std::fabs(b[e]));
            rep.push_back(b);
            rep_scale.push_back(sc);
            found = static_cast<int>(rep.size()) - 1;
        }
        dev = std::max(dev, fdev);
        tag[t] = found;
    }
    M.dm_table.assign(9 * rep.size(), 0.0f);
    for (size_t k = 0; k < rep.size(); ++k)
        for (int e = 0; e < 9; ++e) M.dm_table[9 * k + e] = rep[k][e];
    for (size_t t = 0; t < ns; ++t)
        if (tag[t] >= 0) M.lconn[t] |= dm_type_bits(tag[t]);
    M.dm_dev = dev;
    return true;
}

bool build_pad_mesh(int nv, int nt, int nf, int nm, const float* rest, const int* tets,
                    const int* fixed, const float* markers, int marker_mode, PadMesh& M, std::string& err) {
    if (nv <= 0 || nt <= 0 || nf < 0 || nm < 0 || !rest || !tets || (nf && !fixed) || (nm && !markers)) {
        err = "pad descriptor has a non-positive size or a null array";
        return false;
    }
    if (nv > kVertMask) {
        err = "pad has too many vertices";
        return false;
    }
    M.n_v = nv;
    M.n_t = nt;
    M.n_mk = nm;
    M.X.assign(rest, rest + 3 * static_cast<size_t>(nv));
    M.fixed.assign(nv, 0);
    for (int i = 0; i < nf; ++i) {
        if (fixed[i] < 0 || fixed[i] >= nv) {
            err = "fixed vertex id out of range";
            return false;
        }
        M.fixed[fixed[i]] = 1;
    }
    // rest shape per input tet
    std::vector<double> Binv(9 * static_cast<size_t>(nt));
    std::vector<double> vol(nt);
    M.vlump.assign(nv, 0.0f);
    std::vector<double> vl(nv, 0.0);
    for (int t = 0; t < nt; ++t) {
        const int* c = tets + 4 * static_cast<size_t>(t);
        for (int k = 0; k < 4; ++k)
            if (c[k] < 0 || c[k] >= nv) {
                std::snprintf(msgbuf, sizeof msgbuf, "tet %d has a vertex id out of range", t);
                err = msgbuf;
                return false;
            }
        double Dm[9];
        for (int col = 0; col < 3; ++col)
            for (int r = 0; r < 3; ++r)
                Dm[3 * r + col] = static_cast<double>(rest[3 * c[col + 1] + r]) - static_cast<double>(rest[3 * c[0] + r]);
        double d = det3(Dm);
        if (!(d > 0.0)) {
            std::snprintf(msgbuf, sizeof msgbuf, "tet %d has non-positive rest volume", t);
            err = msgbuf;
            return false;
        }
        inv3(Dm, &Binv[9 * static_cast<size_t>(t)]);
        vol[t] = d / 6.0;
        for (int k = 0; k < 4; ++k) vl[c[k]] += vol[t] / 4.0;
    }
    for (int i = 0; i < nv; ++i) M.vlump[i] = static_cast<float>(vl[i]);
    {
        // b_k = row k-1 of Dm^-1 for corners 1..3, b_0 = -(sum of the rows)
        std::vector<double> wd(nv, 0.0);
        for (int t = 0; t < nt; ++t) {
            const int* c = tets + 4 * static_cast<size_t>(t);
            const double* Bi = &Binv[9 * static_cast<size_t>(t)];
            double b0[3] = {-(Bi[0] + Bi[3] + Bi[6]), -(Bi[1] + Bi[4] + Bi[7]), -(Bi[2] + Bi[5] + Bi[8])};
            wd[c[0]] += vol[t] * (b0[0] * b0[0] + b0[1] * b0[1] + b0[2] * b0[2]);
            for (int k = 1; k < 4; ++k) {
                const double* r = Bi + 3 * (k - 1);
                wd[c[k]] += vol[t] * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            }
        }
        M.wdiag.assign(nv, 0.0f);
        for (int i = 0; i < nv; ++i) M.wdiag[i] = static_cast<float>(wd[i]);
    }

    // canonical surface: boundary faces (sorted ids), sorted lexicographically
    std::vector<std::array<int, 3>> faces;
    faces.reserve(4 * static_cast<size_t>(nt));
    static const int fidx[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    for (int t = 0; t < nt; ++t) {
        const int* c = tets + 4 * static_cast<size_t>(t);
        for (auto& f : fidx) {
            std::array<int, 3> a = {c[f[0]], c[f[1]], c[f[2]]};
            std::sort(a.begin(), a.end());
            faces.push_back(a);
        }
    }
    std::sort(faces.begin(), faces.end());
    std::vector<std::array<int, 3>> surf;
    for (size_t i = 0; i < faces.size();) {
        size_t j = i;
        while (j < faces.size() && faces[j] == faces[i]) ++j;
        if (j - i == 1) surf.push_back(faces[i]);
        i = j;
    }
    M.st.clear();
    std::vector<std::array<int, 2>> edges;
    for (auto& f : surf) {
        M.st.insert(M.st.end(), f.begin(), f.end());
        edges.push_back({f[0], f[1]});
        edges.push_back({f[1], f[2]});
        edges.push_back({f[0], f[2]});
    }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    M.se.clear();
    double lsum = 0.0;
    for (auto& e : edges) {
        M.se.push_back(e[0]);
        M.se.push_back(e[1]);
        double l2 = 0.0;
        for (int r = 0; r < 3; ++r) {
            double dd = static_cast<double>(rest[3 * e[1] + r]) - rest[3 * e[0] + r];
            l2 += dd * dd;
        }
        lsum += std::sqrt(l2);
    }
    M.lbar = edges.empty() ? 0.0 : lsum / edges.size();
    M.sv.clear();
    for (int v : M.st) M.sv.push_back(v);
    std::sort(M.sv.begin(), M.sv.end());
    M.sv.erase(std::unique(M.sv.begin(), M.sv.end()), M.sv.end());

    if (!build_marker_map(nv, rest, M.st, nm, markers, marker_mode, M.mk_ids, M.mk_w, err)) return false;

    // Morton codes on the rest bounding box (10 bits per axis)
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < nv; ++i)
        for (int r = 0; r < 3; ++r) {
            lo[r] = std::min(lo[r], static_cast<double>(rest[3 * i + r]));
            hi[r] = std::max(hi[r], static_cast<double>(rest[3 * i + r]));
        }
    double span = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    auto morton = [&](const double q[3]) {
        uint32_t b[3];
        for (int r = 0; r < 3; ++r) {
            double u = span > 0 ? (q[r] - lo[r]) / span : 0.0;
            b[r] = static_cast<uint32_t>(std::min(1023.0, std::max(0.0, u * 1023.0)));
        }
        return (spread10(b[0]) << 2) | (spread10(b[1]) << 1) | spread10(b[2]);
    };

    // patches: tets in Morton order of their centroids, cut greedily so that a
    // patch has at most kPatchTets tets and kPatchVerts distinct vertices, then
    // coloured so that patches of one colour share no vertex
    std::vector<uint32_t> code(nt);
    for (int t = 0; t < nt; ++t) {
        const int* c = tets + 4 * static_cast<size_t>(t);
        double q[3];
        for (int r = 0; r < 3; ++r)
            q[r] = 0.25 * (rest[3 * c[0] + r] + rest[3 * c[1] + r] + rest[3 * c[2] + r] + rest[3 * c[3] + r]);
        code[t] = morton(q);
    }
    M.tet_order.resize(nt);
    std::iota(M.tet_order.begin(), M.tet_order.end(), 0);
    std::stable_sort(M.tet_order.begin(), M.tet_order.end(), [&](int a, int b) { return code[a] < code[b]; });

    // 1. greedy patches in Morton order (at most kPatchTets tets, kPatchVerts vertices)
    std::vector<std::vector<int>> ptets, pverts;
    {
        std::vector<int> mark(nv, -1);
        std::vector<int> cur_t, cur_v;
        int pid = 0;
        for (int k = 0; k < nt; ++k) {
            const int* c = tets + 4 * static_cast<size_t>(M.tet_order[k]);
            int add = 0;
            for (int j = 0; j < 4; ++j) {
                bool seen = mark[c[j]] == pid;
                for (int jj = 0; jj < j; ++jj) seen = seen || (c[jj] == c[j]);
                add += seen ? 0 : 1;
            }
            if (static_cast<int>(cur_t.size()) >= kPatchTets || static_cast<int>(cur_v.size()) + add > kPatchVerts) {
                ptets.push_back(cur_t);
                pverts.push_back(cur_v);
                cur_t.clear();
                cur_v.clear();
                ++pid;
            }
            cur_t.push_back(M.tet_order[k]);
            for (int j = 0; j < 4; ++j)
                if (mark[c[j]] != pid) {
                    mark[c[j]] = pid;
                    cur_v.push_back(c[j]);
                }
        }
        if (!cur_t.empty()) {
            ptets.push_back(cur_t);
            pverts.push_back(cur_v);
        }
    }
    const int np0 = static_cast<int>(ptets.size());

    // internal vertex order: first appearance along the patches in creation
    // (spatial) order, so that the vertices of a patch lie close together in
    // every per-vertex array. Everything stored from here on uses internal
    // ids; the surface lists and the marker triangles keep the order they
    // have in input ids.
    std::vector<int> vint(nv, -1);
    {
        int next = 0;
        for (int q = 0; q < np0; ++q)
            for (int v : pverts[q])
                if (vint[v] < 0) vint[v] = next++;
        for (int v = 0; v < nv; ++v)
            if (vint[v] < 0) {
                std::snprintf(msgbuf, sizeof msgbuf, "vertex %d belongs to no tet", v);
                err = msgbuf;
                return false;
            }
    }
    M.vuser.assign(nv, 0);
    for (int v = 0; v < nv; ++v) M.vuser[vint[v]] = v;
    {
        std::vector<float> X2(3 * static_cast<size_t>(nv)), vl2(nv), wd2(nv);
        std::vector<uint8_t> fx2(nv);
        for (int j = 0; j < nv; ++j) {
            int u = M.vuser[j];
            for (int r = 0; r < 3; ++r) X2[3 * j + r] = M.X[3 * u + r];
            vl2[j] = M.vlump[u];
            wd2[j] = M.wdiag[u];
            fx2[j] = M.fixed[u];
        }
        M.X.swap(X2);
        M.vlump.swap(vl2);
        M.wdiag.swap(wd2);
        M.fixed.swap(fx2);
    }
    for (int& v : M.sv) v = vint[v];
    for (int& v : M.st) v = vint[v];
    for (int& v : M.se) v = vint[v];
    for (int& v : M.mk_ids) v = vint[v];
    for (auto& pv : pverts)
        for (int& v : pv) v = vint[v];
    std::vector<int> itets(4 * static_cast<size_t>(nt));
    for (size_t k = 0; k < itets.size(); ++k) itets[k] = vint[tets[k]];
    // 2. colour the patches: two patches sharing a vertex get different colours
    std::vector<std::vector<int>> vpatch(nv);
    for (int q = 0; q < np0; ++q)
        for (int v : pverts[q]) vpatch[v].push_back(q);
    std::vector<int> colour(np0, -1);
    int ncol = 0;
    {
        std::vector<int> used(64, -1);
        for (int q = 0; q < np0; ++q) {
            for (int v : pverts[q])
                for (int o : vpatch[v])
                    if (colour[o] >= 0) {
                        if (colour[o] >= static_cast<int>(used.size())) used.resize(colour[o] + 1, -1);
                        used[colour[o]] = q;
                    }
            int c = 0;
            while (c < static_cast<int>(used.size()) && used[c] == q) ++c;
            colour[q] = c;
            ncol = std::max(ncol, c + 1);
        }
    }
    // 2b. balance the classes: the scatter passes process a class in rounds of
    // kCtaWarps patches (one per warp) and end it with a CTA barrier, so a
    // class costs ceil(size / kCtaWarps) rounds. A class whose last round is
    // partly filled moves the patches of that round into classes with free
    // slots in their own last round (where none of the patch's vertices is
    // used); the moves are kept only when all of them succeed, which saves
    // one round each time. Classes left empty disappear.
    {
        const int W = kCtaWarps;
        std::vector<int> size(ncol, 0);
        for (int q = 0; q < np0; ++q) size[colour[q]]++;
        auto fits = [&](int q, int c) {
            for (int v : pverts[q])
                for (int o : vpatch[v])
                    if (o != q && colour[o] == c) return false;
            return true;
        };
        for (bool changed = true; changed;) {
            changed = false;
            std::vector<int> cls(ncol);
            std::iota(cls.begin(), cls.end(), 0);
            std::stable_sort(cls.begin(), cls.end(), [&](int x, int y) { return size[x] < size[y]; });
            for (int a : cls) {
                const int r = size[a] % W;
                if (size[a] == 0 || r == 0) continue;
                std::vector<int> mem;
                for (int q = np0 - 1; q >= 0; --q)
                    if (colour[q] == a) mem.push_back(q);
                std::vector<int> moved;
                for (int q : mem) {
                    if (static_cast<int>(moved.size()) == r) break;
                    for (int c = 0; c < ncol; ++c) {
                        if (c == a || size[c] == 0 || size[c] % W == 0 || !fits(q, c)) continue;
                        colour[q] = c;
                        size[c]++;
                        size[a]--;
                        moved.push_back(q);
                        break;
                    }
                }
                if (static_cast<int>(moved.size()) < r) {
                    for (int q : moved) {
                        size[colour[q]]--;
                        colour[q] = a;
                        size[a]++;
                    }
                } else {
                    changed = true;
                }
            }
        }
        // renumber the classes left, largest first (ties by old index)
        std::vector<int> cls;
        for (int c = 0; c < ncol; ++c)
            if (size[c] > 0) cls.push_back(c);
        std::stable_sort(cls.begin(), cls.end(), [&](int x, int y) { return size[x] > size[y]; });
        std::vector<int> ren(ncol, -1);
        for (size_t k = 0; k < cls.size(); ++k) ren[cls[k]] = static_cast<int>(k);
        for (int q = 0; q < np0; ++q) colour[q] = ren[colour[q]];
        ncol = static_cast<int>(cls.size());
    }
    // 3. patches in colour-major order; tets laid out in that order
    std::vector<int> porder(np0);
    std::iota(porder.begin(), porder.end(), 0);
    std::stable_sort(porder.begin(), porder.end(), [&](int a, int b) { return colour[a] < colour[b]; });
    M.colour_off.assign(ncol + 1, 0);
    for (int q = 0; q < np0; ++q) M.colour_off[colour[q] + 1]++;
    for (int c = 0; c < ncol; ++c) M.colour_off[c + 1] += M.colour_off[c];

    const size_t nsl = static_cast<size_t>(np0) * kPatchTets;
    M.B.assign(9 * nsl, 0.0f);
    M.lconn.assign(nsl, kNoTet);
    M.slot.assign(nsl, 0);
    M.tet_order.assign(nsl, -1);
    M.patch.clear();
    M.pvert.assign(static_cast<size_t>(np0) * kPatchVerts, -1);
    M.pcsr.assign(static_cast<size_t>(np0) * kPatchCsr, 0);
    std::vector<int> local(nv, -1);
    std::vector<int> first_patch(nv, -1), last_patch(nv, -1);
    for (int pi = 0; pi < np0; ++pi) {
        const std::vector<int>& tl = ptets[porder[pi]];
        std::vector<int> verts = pverts[porder[pi]];
        std::sort(verts.begin(), verts.end());        // local ids follow mesh ids
        for (size_t l = 0; l < verts.size(); ++l) local[verts[l]] = static_cast<int>(l);
        int nloc = static_cast<int>(verts.size());
        int ntl = static_cast<int>(tl.size());
        // corner slots: for each local vertex, its (tet, corner) pairs in (tet, corner) order
        std::vector<int> count(kPatchCsr, 0);
        for (int t : tl) {
            const int* c = itets.data() + 4 * static_cast<size_t>(t);
            for (int j = 0; j < 4; ++j) count[local[c[j]] + 1]++;
        }
        for (int l = 0; l < kPatchVerts; ++l) count[l + 1] += count[l];   // unused entries: empty runs
        std::vector<int> cursor(count.begin(), count.end() - 1);
        const int csr_begin = pi * kPatchCsr;
        for (int l = 0; l < kPatchCsr; ++l) M.pcsr[csr_begin + l] = static_cast<uint16_t>(count[l]);
        const int tb = pi * kPatchTets;
        for (int k = 0; k < ntl; ++k) {
            const int t = tl[k];
            const int* c = itets.data() + 4 * static_cast<size_t>(t);
            uint32_t lc = 0, sl = 0;
            for (int j = 0; j < 4; ++j) {
                int l = local[c[j]];
                lc |= static_cast<uint32_t>(l) << (8 * j);
                sl |= static_cast<uint32_t>(cursor[l]++) << (8 * j);
            }
            M.lconn[tb + k] = lc;
            M.slot[tb + k] = sl;
            M.tet_order[tb + k] = t;
            for (int e = 0; e < 9; ++e)
                M.B[static_cast<size_t>(e) * nsl + tb + k] = static_cast<float>(Binv[9 * static_cast<size_t>(t) + e]);
        }
        const int vert_begin = pi * kPatchVerts;
        for (int l = 0; l < nloc; ++l) {
            int v = verts[l];
            M.pvert[vert_begin + l] = v;
            if (first_patch[v] < 0) first_patch[v] = pi;
            last_patch[v] = pi;
            local[v] = -1;
        }
        M.patch.push_back(tb);
        M.patch.push_back(vert_begin);
        M.patch.push_back(ntl | (nloc << 16));
        M.patch.push_back(csr_begin);
    }
    // first / last flags (processing order: colour-major)
    int np = M.n_patch();
    for (int p = 0; p < np; ++p) {
        int vb = M.patch[4 * p + 1], nl = M.patch[4 * p + 2] >> 16;
        for (int l = 0; l < nl; ++l) {
            int v = M.pvert[vb + l];
            if (first_patch[v] == p) M.pvert[vb + l] |= kFirstFlag;
            if (last_patch[v] == p) M.pvert[vb + l] |= kLastFlag;
        }
    }
    for (int v = 0; v < nv; ++v)
        if (first_patch[v] < 0) {
            std::snprintf(msgbuf, sizeof msgbuf, "vertex %d belongs to no tet", M.vuser[v]);
            err = msgbuf;
            return false;
        }
    return true;
}

bool build_indenter_mesh(int nv, int nt, const float* verts, const int* tris, IndenterMesh& I,
                         std::string& err) {
    if (nv <= 0 || nt <= 0 || !verts || !tris) {
        err = "indenter descriptor has a non-positive size or a null array";
        return false;
    }
    I.n_v = nv;
    I.n_t = nt;
    I.Y.assign(verts, verts + 3 * static_cast<size_t>(nv));
    I.tris.assign(tris, tris + 3 * static_cast<size_t>(nt));
    std::vector<std::array<int, 2>> e;
    for (int t = 0; t < nt; ++t) {
        int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= nv || b >= nv || c >= nv) {
            err = "indenter triangle has a vertex id out of range";
            return false;
        }
        e.push_back({std::min(a, b), std::max(a, b)});
        e.push_back({std::min(b, c), std::max(b, c)});
        e.push_back({std::min(a, c), std::max(a, c)});
    }
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    I.n_e = static_cast<int>(e.size());
    I.edges.clear();
    for (auto& x : e) {
        I.edges.push_back(x[0]);
        I.edges.push_back(x[1]);
    }
    return true;
}

}  // namespace tac
