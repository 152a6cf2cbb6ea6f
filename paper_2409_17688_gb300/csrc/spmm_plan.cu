// Host-side plan builder of the sparse (min,+) step (K2): row groups, their
// unions and stages, row clusters and membership-mask segments, the per-warp
// entry streams of every stage's blob, and each CTA's unit schedule.  The
// kernel that walks the plan is in spmm.cu; the plan's format is described
// there and in spmm.cuh.
#include <algorithm>
#include <cstring>
#include <iterator>

#include "spmm.cuh"

namespace mp {

int plan_build_host(const HostCsr &csr, bool colconst, const std::vector<uint16_t> &z,
                    const std::vector<int32_t> *canon, int64_t ncols,
                    int cap_rows, int blob_cap, int grid, PlanHost *out, int cluster_max) {
    const int64_t N = csr.N;
    if (ncols <= 0) ncols = N;
    const int umax = cap_rows - 1;  // the last buffer row is the INF padding row
    if (umax < 1) return set_error(MP_EINVAL, "shared-memory buffer too small");
    if ((int64_t)cap_rows * kRowBytes > (int64_t)kEntOffset + 1)
        return set_error(MP_EINVAL, "%d buffer rows exceed the entry offset field", cap_rows);
    PlanHost &P = *out;
    P = PlanHost();
    P.N = N;
    P.colconst = colconst;
    P.cap_rows = cap_rows;
    P.blob_cap = blob_cap;
    P.z = z;
    if (P.z.size() != (size_t)N) P.z.assign((size_t)N, 0);
    P.ldb = ((ncols + kChunk - 1) / kChunk) * kChunk;
    P.nchunks = (int)(P.ldb / kChunk);
    P.nnz = csr.row_ptr[N];

    const int per_entry = colconst ? 1 : 2;  // 32-bit words per entry
    const int pad_to = colconst ? 8 : 4;     // entries per pass of the gather loop
    const int gran = pad_to * per_entry;     // words a segment's length is a multiple of
    auto padded = [&](int64_t cnt) { return (cnt + pad_to - 1) / pad_to * pad_to; };
    auto blob_words = [&](int64_t rows, int64_t entry_words) {
        const int64_t labels = ((rows + 15) / 16) * 8 + ((rows + 7) & ~7);  // z, caller rows
        if (colconst)  // task words, labels, entry streams
            return (int64_t)kBlobHeader + ((rows + kWarps + 7) & ~7) + labels + entry_words;
        return (int64_t)kBlobHeader + ((2 * (rows + kWarps) + 7) & ~7) +
               ((2 * (15 * rows + 2 * kWarps) + 7) & ~7) + labels + entry_words;
    };

    std::vector<int32_t> stamp((size_t)N, -1), local((size_t)N, -1);
    P.grp_row0.push_back(0);
    P.grp_stage0.push_back(0);
    P.stage_u0.push_back(0);
    P.blob_off.push_back(0);
    int32_t gid = 0, attempt = 0;
    // When rows are long against the buffer (mean length above a quarter of
    // it) a one-buffer union holds only a few rows and every gathered row is
    // staged again for each of those small groups.  Such matrices get groups
    // whose union spans up to kStagesMax buffers: more rows share each staged
    // row, and the stages' minima carry over in the shared accumulators.
    const bool long_rows = N > 0 && 4 * csr.row_ptr[N] > (int64_t)umax * N;
    const int64_t u_limit = long_rows ? (int64_t)kStagesMax * umax : umax;
    int64_t q = 0;
    while (q < N) {
        // grow the group while the union of gathered rows fits its stages and
        // a stage's entry blob fits the blob region (estimated from the rows'
        // lengths shared out over the stages; a stage that still overflows is
        // rebuilt with fewer rows below)
        const int64_t g0 = q;
        int64_t ucount = 0, ewords = 0;
        while (q < N && q - g0 < kGroupMax) {
            int64_t add = 0;
            for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e)
                if (stamp[csr.col[e]] != gid) ++add;
            const int64_t ew = padded(csr.row_ptr[q + 1] - csr.row_ptr[q]) * per_entry;
            const int64_t nst = std::max<int64_t>(1, (ucount + add + umax - 1) / umax);
            if (q > g0 && (ucount + add > u_limit ||
                           blob_words(q - g0 + 1, (ewords + ew) / nst) > blob_cap))
                break;
            for (int64_t e = csr.row_ptr[q]; e < csr.row_ptr[q + 1]; ++e) stamp[csr.col[e]] = gid;
            ucount += add;
            ewords += ew;
            ++q;
        }
        // Build the group's stages; if a stage's blob overflows its region
        // (mask padding of the clusters can exceed the row-wise estimate),
        // retry with fewer rows.
        int64_t qend = q;
        while (true) {
            const size_t snap_urows = P.urows.size(), snap_su = P.stage_u0.size();
            const size_t snap_blob = P.blob.size(), snap_bo = P.blob_off.size();
            bool overflow = false;
            ++attempt;
            // the union, sorted, cut into stages of at most umax rows
            std::vector<int32_t> U;
            U.reserve((size_t)ucount);
            for (int64_t r = g0; r < qend; ++r)
                for (int64_t e = csr.row_ptr[r]; e < csr.row_ptr[r + 1]; ++e)
                    if (local[csr.col[e]] != attempt) {
                        local[csr.col[e]] = attempt;
                        U.push_back(csr.col[e]);
                    }
            std::sort(U.begin(), U.end());
            const int nst = U.empty() ? 1 : (int)((U.size() + umax - 1) / umax);
            for (int st = 0; st < nst; ++st) {
                const size_t ub = (size_t)st * umax, ue = std::min(U.size(), ub + (size_t)umax);
                for (size_t u = ub; u < ue; ++u) P.urows.push_back(U[u]);
                P.stage_u0.push_back((int32_t)P.urows.size());
                const int64_t rows = qend - g0;
                // gathered-row indices (local to the stage) of every row of the group
                std::vector<std::vector<int32_t>> rloc((size_t)rows);
                std::vector<std::vector<uint32_t>> rval((size_t)rows);
                for (int64_t r = g0; r < qend; ++r) {
                    std::vector<std::pair<int32_t, uint32_t>> es;
                    for (int64_t e = csr.row_ptr[r]; e < csr.row_ptr[r + 1]; ++e) {
                        const int32_t p = csr.col[e];
                        const size_t u = (size_t)(std::lower_bound(U.begin(), U.end(), p) - U.begin());
                        if (u < ub || u >= ue) continue;
                        es.push_back({(int32_t)(u - ub), (uint32_t)(uint16_t)csr.val[e]});
                    }
                    std::sort(es.begin(), es.end());
                    for (auto &pr : es) {
                        rloc[r - g0].push_back(pr.first);
                        rval[r - g0].push_back(pr.second);
                    }
                }
                // clusters: with one label per gathered row (column-constant A)
                // rows whose gather lists overlap share the reads; greedy clusters
                // of up to cluster_max (at most 4) rows, each next row the one
                // overlapping most
                std::vector<std::vector<int>> clusters;
                {
                    std::vector<int> rem;
                    for (int r = 0; r < (int)rows; ++r)
                        if (!rloc[r].empty()) rem.push_back(r);
                    auto overlap = [&](const std::vector<int32_t> &x, const std::vector<int32_t> &y) {
                        size_t i = 0, j = 0, c = 0;
                        while (i < x.size() && j < y.size()) {
                            if (x[i] < y[j]) ++i;
                            else if (y[j] < x[i]) ++j;
                            else { ++c; ++i; ++j; }
                        }
                        return c;
                    };
                    const int kmax = colconst ? std::max(1, std::min(4, cluster_max)) : 1;
                    while (!rem.empty()) {
                        std::vector<int> cl{rem.front()};
                        rem.erase(rem.begin());
                        std::vector<int32_t> inter = rloc[cl[0]];
                        while ((int)cl.size() < kmax && !rem.empty()) {
                            size_t best = 0, bi = 0;
                            for (size_t k = 0; k < rem.size(); ++k) {
                                const size_t ov = overlap(inter, rloc[rem[k]]);
                                if (ov > best) { best = ov; bi = k; }
                            }
                            if (best == 0) break;
                            const int nxt = rem[bi];
                            rem.erase(rem.begin() + (long)bi);
                            std::vector<int32_t> ni;
                            std::set_intersection(inter.begin(), inter.end(), rloc[nxt].begin(),
                                                  rloc[nxt].end(), std::back_inserter(ni));
                            inter.swap(ni);
                            cl.push_back(nxt);
                        }
                        clusters.push_back(cl);
                    }
                }
                // per cluster: its union split by membership mask into segments of
                // entries (padded to whole unrolled iterations)
                struct Seg { int mask; std::vector<uint32_t> words; };
                struct Cl { std::vector<int> rows; std::vector<Seg> segs; int64_t words = 0; };
                std::vector<Cl> cls;
                for (auto &cl : clusters) {
                    Cl c;
                    c.rows = cl;
                    std::vector<std::pair<int32_t, std::pair<int, uint32_t>>> all;  // (u, (row j, label))
                    for (int j = 0; j < (int)cl.size(); ++j)
                        for (size_t t = 0; t < rloc[cl[j]].size(); ++t)
                            all.push_back({rloc[cl[j]][t], {j, rval[cl[j]][t]}});
                    std::sort(all.begin(), all.end());
                    std::vector<std::vector<std::pair<int32_t, uint32_t>>> bym(16);
                    for (size_t i = 0; i < all.size();) {
                        size_t k = i;
                        int mask = 0;
                        while (k < all.size() && all[k].first == all[i].first) mask |= 1 << all[k++].second.first;
                        bym[mask].push_back({all[i].first, all[i].second.second});
                        i = k;
                    }
                    for (int mask = 1; mask < 16; ++mask) {
                        auto &v = bym[mask];
                        if (v.empty()) continue;
                        while (v.size() % pad_to) v.push_back({umax, 0u});  // padding row
                        Seg sg;
                        sg.mask = mask;
                        for (auto &pr : v) {
                            sg.words.push_back((uint32_t)pr.first * kRowBytes);
                            if (!colconst) sg.words.push_back(pr.second * 0x10001u);
                        }
                        c.words += (int64_t)sg.words.size();
                        c.segs.push_back(std::move(sg));
                    }
                    cls.push_back(std::move(c));
                }
                // Entries laid out cluster by cluster, and that sequence cut into
                // at most kWarps contiguous ranges of equal cost, one per warp: a
                // cluster that straddles a cut becomes two tasks.  A range's cost counts, besides its entry words, the
                // work at each segment end and at each task end, in entry words.
                const int64_t seg_cost = 12 * per_entry, task_cost = 32 * per_entry;
                int64_t total = 0;
                for (auto &c : cls) total += c.words + seg_cost * (int64_t)c.segs.size() + task_cost;
                struct SegRef { int mask; int64_t e0, e1; };
                struct Task { int ci; std::vector<SegRef> segs; int64_t len; };
                std::vector<Task> tasks;
                std::vector<uint32_t> ents;
                std::vector<std::vector<int>> per_warp(kWarps);
                // each cut adds a task end and a segment end; small units use
                // fewer warps so that a range costs at least twice that
                const int64_t cut_cost = task_cost + seg_cost;
                int nw = kWarps;
                while (nw > 1 && total + (nw - 1) * cut_cost < 2 * cut_cost * nw) --nw;
                const int64_t whole = total + (nw - 1) * cut_cost;
                int cw = 0;
                int64_t spent = 0;
                auto bound = [&](int w) { return (w + 1) * whole / nw; };
                for (int ci = 0; ci < (int)cls.size(); ++ci) {
                    Task cur{ci, {}, 0};
                    spent += task_cost;
                    for (auto &sg : cls[ci].segs) {
                        int64_t e = (int64_t)ents.size();
                        ents.insert(ents.end(), sg.words.begin(), sg.words.end());
                        const int64_t end = (int64_t)ents.size();
                        while (e < end) {
                            int64_t take = end - e;
                            if (cw < nw - 1) {
                                const int64_t room = bound(cw) - spent - seg_cost;
                                take = std::min(take, std::max<int64_t>(gran, (room + gran - 1) / gran * gran));
                            }
                            cur.segs.push_back({sg.mask, e, e + take});
                            cur.len += take;
                            spent += take + seg_cost;
                            e += take;
                            if (cw < nw - 1 && spent >= bound(cw)) {
                                tasks.push_back(cur);
                                per_warp[cw++].push_back((int)tasks.size() - 1);
                                cur = Task{ci, {}, 0};
                                spent += task_cost;
                            }
                        }
                    }
                    if (!cur.segs.empty()) {
                        tasks.push_back(cur);
                        per_warp[cw].push_back((int)tasks.size() - 1);
                    }
                }
                int nsegs = 0;
                for (auto &t : tasks) nsegs += (int)t.segs.size();
                const int ntasks = (int)tasks.size();
                std::vector<uint32_t> blob((size_t)kBlobHeader, 0u);
                blob[0] = (uint32_t)g0;
                blob[1] = (uint32_t)rows;
                blob[2] = (st == 0 ? 1u : 0u) | (st == nst - 1 ? 2u : 0u);
                blob[3] = (uint32_t)ntasks;
                blob[4] = (uint32_t)nsegs;
                auto task_word = [&](const Task &t) {
                    const auto &cr = cls[t.ci].rows;
                    uint32_t w0 = (uint32_t)cr.size() << 24;
                    for (int j = 0; j < (int)cr.size(); ++j) w0 |= (uint32_t)cr[j] << (6 * j);
                    return w0;
                };
                // labels of the group's rows (16-bit), added when a row is written
                std::vector<uint32_t> zw((size_t)((rows + 15) / 16) * 8, 0u);
                for (int64_t r = 0; r < rows; ++r)
                    zw[(size_t)(r >> 1)] |= (uint32_t)P.z[(size_t)(g0 + r)] << (16 * (r & 1));
                // then the caller's row of each group row (where its values and
                // diagonal entry go), 32-bit, padded to 8 words
                for (int64_t r = 0; r < ((rows + 7) & ~7); ++r)
                    zw.push_back(r < rows ? (uint32_t)(canon ? (*canon)[(size_t)(g0 + r)] : g0 + r) : 0u);
                int tcount = 0;
                if (colconst) {
                    // per warp: its tasks' entries back to back, segment and task
                    // ends flagged in the last entry word, padded to 8-entry blocks
                    std::vector<uint32_t> ttab, stream;
                    for (int wv = 0; wv < kWarps; ++wv) {
                        blob[8 + wv] = (uint32_t)tcount;
                        blob[kStreamStart + wv] = (uint32_t)stream.size();
                        for (int ti : per_warp[wv]) {
                            const Task &t = tasks[ti];
                            ttab.push_back(task_word(t));
                            ++tcount;
                            for (size_t k = 0; k < t.segs.size(); ++k) {
                                const SegRef &sr = t.segs[k];
                                stream.insert(stream.end(), ents.begin() + sr.e0, ents.begin() + sr.e1);
                                const uint32_t f = kEntSegEnd | ((uint32_t)sr.mask << kEntMaskShift) |
                                                   (k + 1 == t.segs.size() ? kEntTaskEnd : 0u);
                                for (size_t i = stream.size() - 4; i < stream.size(); ++i) stream[i] |= f;
                            }
                        }
                    }
                    blob[8 + kWarps] = (uint32_t)tcount;
                    blob[kStreamStart + kWarps] = (uint32_t)stream.size();
                    ttab.resize((size_t)((ntasks + 7) & ~7), 0u);
                    blob.insert(blob.end(), ttab.begin(), ttab.end());
                    blob.insert(blob.end(), zw.begin(), zw.end());
                    blob.insert(blob.end(), stream.begin(), stream.end());
                } else {
                    std::vector<uint32_t> ttab((size_t)((2 * ntasks + 7) & ~7), 0u);
                    std::vector<uint32_t> stab((size_t)((2 * nsegs + 7) & ~7), 0u);
                    int scount = 0;
                    for (int wv = 0; wv < kWarps; ++wv) {
                        blob[8 + wv] = (uint32_t)tcount;
                        for (int ti : per_warp[wv]) {
                            const Task &t = tasks[ti];
                            ttab[2 * tcount] = task_word(t);
                            ttab[2 * tcount + 1] =
                                (uint32_t)scount | ((uint32_t)(scount + t.segs.size()) << 16);
                            for (auto &sr : t.segs) {
                                stab[2 * scount] = (uint32_t)sr.e0 | ((uint32_t)sr.mask << 16);
                                stab[2 * scount + 1] = (uint32_t)sr.e1;
                                ++scount;
                            }
                            ++tcount;
                        }
                    }
                    blob[8 + kWarps] = (uint32_t)tcount;
                    blob.insert(blob.end(), ttab.begin(), ttab.end());
                    blob.insert(blob.end(), stab.begin(), stab.end());
                    blob.insert(blob.end(), zw.begin(), zw.end());
                    blob.insert(blob.end(), ents.begin(), ents.end());
                }
                while (blob.size() % 8) blob.push_back(0u);  // 32-byte granules for the copy
                if ((int64_t)ents.size() > 0xFFFF || nsegs > 0xFFFF)
                    return set_error(MP_EINVAL, "stage entry list of %zu words too long", ents.size());
                if ((int64_t)blob.size() > blob_cap) {
                    overflow = true;
                    break;
                }
                P.blob.insert(P.blob.end(), blob.begin(), blob.end());
                P.blob_off.push_back((int64_t)P.blob.size());
            }
            if (!overflow) break;
            if (qend - g0 == 1)
                return set_error(MP_EINVAL, "a single row's stage blob exceeds the %d-word region",
                                 blob_cap);
            P.urows.resize(snap_urows);
            P.stage_u0.resize(snap_su);
            P.blob.resize(snap_blob);
            P.blob_off.resize(snap_bo);
            qend = g0 + std::max<int64_t>(1, (qend - g0) * 3 / 4);
        }
        q = qend;
        P.grp_row0.push_back((int32_t)q);
        P.grp_stage0.push_back((int32_t)(P.stage_u0.size() - 1));
        ++gid;
    }
    P.ngroups = gid;

    // Schedule: work items (group, chunk) dealt to the CTAs longest first,
    // each CTA's items then ordered by chunk; a unit per stage of an item.
    P.grid = std::max(1, grid);
    if (P.nchunks > 0xFFFF || (int64_t)P.blob.size() / 8 > 0xFFFFFFFFll)
        return set_error(MP_EINVAL, "plan too large for the packed unit descriptors");
    std::vector<int64_t> gcost((size_t)gid, 0);
    for (int gg = 0; gg < gid; ++gg)
        for (int st = P.grp_stage0[gg]; st < P.grp_stage0[gg + 1]; ++st)
            gcost[gg] += (P.blob_off[st + 1] - P.blob_off[st]) + 256;  // entries + fixed cost
    struct Item { int64_t cost; int32_t g, chunk; };
    std::vector<Item> items;
    items.reserve((size_t)gid * P.nchunks);
    for (int c = 0; c < P.nchunks; ++c)
        for (int gg = 0; gg < gid; ++gg) items.push_back({gcost[gg], gg, c});
    std::stable_sort(items.begin(), items.end(),
                     [](const Item &x, const Item &y) { return x.cost > y.cost; });
    std::vector<std::vector<Item>> per_cta((size_t)P.grid);
    std::vector<int64_t> load((size_t)P.grid, 0);
    {
        // least-loaded CTA first (a binary heap of (load, cta))
        std::vector<std::pair<int64_t, int>> heap;
        for (int c = 0; c < P.grid; ++c) heap.push_back({0, c});
        auto cmp = [](const std::pair<int64_t, int> &x, const std::pair<int64_t, int> &y) {
            return x.first > y.first || (x.first == y.first && x.second > y.second);
        };
        std::make_heap(heap.begin(), heap.end(), cmp);
        for (auto &it : items) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto &top = heap.back();
            per_cta[(size_t)top.second].push_back(it);
            top.first += it.cost;
            std::push_heap(heap.begin(), heap.end(), cmp);
        }
    }
    P.cta_unit0.assign((size_t)P.grid + 1, 0);
    for (int c = 0; c < P.grid; ++c) {
        auto &L = per_cta[(size_t)c];
        std::sort(L.begin(), L.end(), [](const Item &x, const Item &y) {
            return x.chunk != y.chunk ? x.chunk < y.chunk : x.g < y.g;
        });
        for (auto &it : L)
            for (int st = P.grp_stage0[it.g]; st < P.grp_stage0[it.g + 1]; ++st) {
                UnitDesc u;
                const int64_t bw = P.blob_off[st + 1] - P.blob_off[st];
                const bool last = st + 1 == P.grp_stage0[it.g + 1];
                u.meta = (uint32_t)it.chunk | ((uint32_t)(bw / 8) << 16) | (last ? 0x80000000u : 0u);
                u.u0 = (uint32_t)P.stage_u0[st];
                u.u1 = (uint32_t)P.stage_u0[st + 1];
                u.bo8 = (uint32_t)(P.blob_off[st] / 8);
                P.units.push_back(u);
            }
        P.cta_unit0[(size_t)c + 1] = (int32_t)P.units.size();
    }
    return MP_OK;
}

}  // namespace mp
