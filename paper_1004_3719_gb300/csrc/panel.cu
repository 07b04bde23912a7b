// Host side of the x-panel layout (FFSPMV_FMT_PANEL): row groups, column
// groups, panels, stages, and the order of the entries inside a stage.
//
// The device kernel (k_panel, kernels.cu) streams each CTA's stages through
// shared memory; what it costs per entry is one shared-memory gather of x and,
// for short rows, one shared-memory atomic into the row's sum.  Both land in
// banks chosen by the data, so this file orders the entries of every 32 lanes
// (one warp instruction per slot) to spread them over the banks:
//   * a row with at least eight entries in a stage gives "packs" of eight,
//     summed by one lane; the lanes of one warp that carry the same row are
//     summed together before a single atomic, and the eight entries of every
//     pack lane are ordered so that each slot's x words fall in distinct banks
//     where possible;
//   * the other entries ("singles") are drawn slot by slot from a pool keyed
//     by (x bank, row-sum bank), greedily taking a bank pair not yet used in
//     the slot and preferring the banks with the most entries left.
// +-1 entries (Sec. 2.4.2) go to sections without values when segregation is
// on; their sign is a bit of the entry word.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>
#include <vector>

#include "ff_internal.cuh"
#include "ff_plan.h"

namespace ff {

namespace {

// One entry of a stage before layout.
struct SEnt {
    u32 row;  // row in the group
    u32 idx;  // x element of the panel
    u32 val;  // residue (general entries; 0 for padding)
    u32 neg;  // +-1 sections: 1 for a -1 entry
};

// Bank of x element idx (xb bytes per column: 1, 2, 4, 8 or 16) and of the row
// sums of a row (ab bytes per row: 4 to 32); wider words are numbered by
// their 4-byte bank group, so that distinct numbers mean distinct banks.
inline int xbank_of(u32 idx, int xb)
{
    return xb == 1 ? (int)((idx >> 2) & 31u) : xb == 2 ? (int)((idx >> 1) & 31u) : (int)(idx % (128u / xb));
}
inline int rbank_of(u32 row, int ab) { return (int)(row % (128u / ab)); }

// Single entries keyed by (x bank, row-sum bank).
struct Pool {
    std::vector<SEnt> e;         // sorted by bucket
    int start[32][32], take[32][32], cnt[32][32];
    int xrem[32], rrem[32];
    long long left = 0;

    void init(const std::vector<SEnt> &in, int xb, int ab)
    {
        memset(start, 0, sizeof start);
        memset(take, 0, sizeof take);
        memset(cnt, 0, sizeof cnt);
        memset(xrem, 0, sizeof xrem);
        memset(rrem, 0, sizeof rrem);
        for (const SEnt &s : in) cnt[xbank_of(s.idx, xb)][rbank_of(s.row, ab)]++;
        int off = 0;
        for (int a = 0; a < 32; ++a)
            for (int b = 0; b < 32; ++b) {
                start[a][b] = off;
                off += cnt[a][b];
                xrem[a] += cnt[a][b];
                rrem[b] += cnt[a][b];
            }
        e.assign(in.size(), SEnt{0, 0, 0, 0});
        int pos[32][32];
        memcpy(pos, start, sizeof pos);
        for (const SEnt &s : in) e[pos[xbank_of(s.idx, xb)][rbank_of(s.row, ab)]++] = s;
        left = (long long)in.size();
    }

    SEnt pop(int a, int b)
    {
        SEnt s = e[start[a][b] + take[a][b]++];
        cnt[a][b]--;
        xrem[a]--;
        rrem[b]--;
        left--;
        return s;
    }
};

// Fill `c` lanes' slot from the pool: x banks distinct and row-sum banks
// distinct at level 1, then at most two per bank, and so on.  mx: x banks
// already used in this slot (by other lanes of the warp).
void fill_slot(Pool &P, int c, int mx[32], int mr[32], std::vector<SEnt> &out)
{
    int order[32];
    std::iota(order, order + 32, 0);
    std::sort(order, order + 32, [&](int a, int b) { return P.xrem[a] > P.xrem[b]; });
    int picked = 0;
    for (int level = 1; picked < c && P.left > 0; ++level) {
        bool progress = true;
        while (progress && picked < c && P.left > 0) {
            progress = false;
            for (int k = 0; k < 32 && picked < c; ++k) {
                const int a = order[k];
                if (mx[a] >= level || P.xrem[a] == 0) continue;
                int best = -1, bv = -1;
                for (int b = 0; b < 32; ++b)
                    if (P.cnt[a][b] > 0 && mr[b] < level && P.rrem[b] > bv) {
                        best = b;
                        bv = P.rrem[b];
                    }
                if (best < 0) continue;
                out.push_back(P.pop(a, best));
                mx[a]++;
                mr[best]++;
                picked++;
                progress = true;
            }
        }
    }
}

// Per-row packs of eight (entries already sorted by row); the rest are singles.
void split_packs(const std::vector<SEnt> &in, std::vector<std::vector<SEnt>> &packs, std::vector<SEnt> &singles)
{
    size_t i = 0;
    while (i < in.size()) {
        size_t j = i;
        while (j < in.size() && in[j].row == in[i].row) ++j;
        const size_t np = (j - i) / 8;
        for (size_t p = 0; p < np; ++p) packs.emplace_back(in.begin() + i + 8 * p, in.begin() + i + 8 * p + 8);
        singles.insert(singles.end(), in.begin() + i + 8 * np, in.begin() + j);
        i = j;
    }
}

// Lays out one stage: writes its entries (and the values of its general
// lanes) and fills the counts of `st`.
void lay_stage(const std::vector<SEnt> &ents, const std::vector<unsigned char> &is_pm, int xb, int ab,
               bool small, std::vector<u32> &ent_out, std::vector<u32> &val_out, PanelStage &st, long long &npad,
               long long &npm)
{
    std::vector<SEnt> gen, pm;
    for (size_t t = 0; t < ents.size(); ++t) (is_pm[t] ? pm : gen).push_back(ents[t]);
    std::vector<std::vector<SEnt>> gpk, ppk;
    std::vector<SEnt> gsg, psg;
    split_packs(gen, gpk, gsg);
    split_packs(pm, ppk, psg);
    // the +-1 singles must fill whole lanes: the odd ones join the general
    // singles with their values (1 or m - 1, already in .val)
    while (psg.size() % 8) {
        gsg.push_back(psg.back());
        gsg.back().neg = 0;
        psg.pop_back();
    }
    if (gsg.size() % 8) {
        const u32 r = gsg.empty() ? 0 : gsg.front().row;
        while (gsg.size() % 8) {
            gsg.push_back(SEnt{r, 0, 0, 0});
            ++npad;
        }
    }
    npm += (long long)(8 * ppk.size() + psg.size());
    const int lpg = (int)gpk.size(), lgs = (int)(gsg.size() / 8), lpp = (int)ppk.size(),
              lps = (int)(psg.size() / 8);
    const int nlg = lpg + lgs, nl = nlg + lpp + lps;
    Pool G, Q;
    G.init(gsg, xb, ab);
    Q.init(psg, xb, ab);
    // lanes: kind 0 general pack, 1 general single, 2 +-1 pack, 3 +-1 single
    auto kind_of = [&](int t) { return t < lpg ? 0 : t < nlg ? 1 : t < nlg + lpp ? 2 : 3; };
    std::vector<std::vector<SEnt>> lane(nl);
    for (int t = 0; t < lpg; ++t) lane[t] = gpk[t];
    for (int t = 0; t < lpp; ++t) lane[nlg + t] = ppk[t];
    for (int b0 = 0; b0 < nl; b0 += 32) {
        const int c = std::min(32, nl - b0);
        // pack lanes: order each pack's eight entries so that every slot's x
        // banks differ across the warp where possible
        std::vector<int> pl, gl, ql;
        for (int t = b0; t < b0 + c; ++t) {
            const int k = kind_of(t);
            (k == 0 || k == 2 ? pl : k == 1 ? gl : ql).push_back(t);
        }
        std::vector<std::vector<SEnt>> rest(pl.size());
        for (size_t i = 0; i < pl.size(); ++i) {
            rest[i] = lane[pl[i]];
            lane[pl[i]].clear();
        }
        std::vector<std::vector<SEnt>> single_slots(8);
        const int cp = (int)pl.size();
        for (int u = 0; u < 8; ++u) {
            int mx[32] = {0}, mr[32] = {0};
            // the pack lanes' entries for this slot: a maximum matching of
            // lanes to distinct x banks (augmenting paths), lanes with the
            // fewest distinct banks first; unmatched lanes take the entry
            // whose bank is least used
            int owner[32], choice[32];
            for (int b = 0; b < 32; ++b) owner[b] = -1;
            for (int i = 0; i < cp; ++i) choice[i] = -1;
            std::vector<int> ord(cp);
            std::iota(ord.begin(), ord.end(), 0);
            std::vector<u32> bankset(cp, 0);
            for (int i = 0; i < cp; ++i)
                for (const SEnt &e : rest[i]) bankset[i] |= 1u << xbank_of(e.idx, xb);
            std::sort(ord.begin(), ord.end(),
                      [&](int a, int b) { return __builtin_popcount(bankset[a]) < __builtin_popcount(bankset[b]); });
            std::function<bool(int, u32 &)> augment = [&](int i, u32 &seen) {
                for (size_t k = 0; k < rest[i].size(); ++k) {
                    const int b = xbank_of(rest[i][k].idx, xb);
                    if (seen & (1u << b)) continue;
                    seen |= 1u << b;
                    if (owner[b] < 0 || augment(owner[b], seen)) {
                        owner[b] = i;
                        choice[i] = (int)k;
                        return true;
                    }
                }
                return false;
            };
            for (int i : ord) {
                u32 seen = 0;
                augment(i, seen);
            }
            // a lane whose matched bank was taken over re-points through owner[]
            for (int i = 0; i < cp; ++i) choice[i] = -1;
            for (int b = 0; b < 32; ++b)
                if (owner[b] >= 0)
                    for (size_t k = 0; k < rest[owner[b]].size(); ++k)
                        if (xbank_of(rest[owner[b]][k].idx, xb) == b) {
                            choice[owner[b]] = (int)k;
                            break;
                        }
            for (int i = 0; i < cp; ++i)
                if (choice[i] >= 0) mx[xbank_of(rest[i][choice[i]].idx, xb)]++;
            for (int i = 0; i < cp; ++i) {
                if (choice[i] < 0) {
                    int best = 0;
                    for (size_t k = 1; k < rest[i].size(); ++k)
                        if (mx[xbank_of(rest[i][k].idx, xb)] < mx[xbank_of(rest[i][best].idx, xb)]) best = (int)k;
                    choice[i] = best;
                    mx[xbank_of(rest[i][best].idx, xb)]++;
                }
                lane[pl[i]].push_back(rest[i][choice[i]]);
                rest[i].erase(rest[i].begin() + choice[i]);
            }
            std::vector<SEnt> &got = single_slots[u];
            fill_slot(G, (int)gl.size(), mx, mr, got);
            fill_slot(Q, (int)ql.size(), mx, mr, got);
        }
        for (int u = 0; u < 8; ++u) {
            for (size_t i = 0; i < gl.size(); ++i) lane[gl[i]].push_back(single_slots[u][i]);
            for (size_t i = 0; i < ql.size(); ++i) lane[ql[i]].push_back(single_slots[u][gl.size() + i]);
        }
    }
    // write out: entries interleaved by four per 32-lane block, values of the
    // general lanes lane by lane (u16) or interleaved like the entries (u32)
    st.k0 = (u32)ent_out.size();
    st.v0 = (u32)val_out.size();
    st.nent = (u32)(8 * nl);
    st.ngen = (u32)(8 * nlg);
    st.npg = (u32)(8 * lpg);
    st.npp = (u32)(8 * lpp);
    ent_out.resize(ent_out.size() + 8 * (size_t)nl);
    // u8 values (xb == 1) are padded to 16 per stage: the bulk copies of a
    // stage's values start and end on 16-byte boundaries
    const size_t vpad = xb == 1 ? 16 : 8;
    val_out.resize((val_out.size() + 8 * (size_t)nlg + vpad - 1) / vpad * vpad);
    for (int t = 0; t < nl; ++t) {
        const int b0 = t / 32 * 32, j = t - b0, c = std::min(32, nl - b0);
        const int cg = std::min(32, nlg - b0);
        const bool general = t < nlg;
        for (int u = 0; u < 8; ++u) {
            const SEnt &s = lane[t][u];
            const int pos = 8 * b0 + (u < 4 ? 4 * j + u : 4 * c + 4 * j + (u - 4));
            ent_out[st.k0 + pos] = (s.row << 16) | ((general ? 0u : s.neg) << 15) | s.idx;
            if (general) {
                const int vpos = small ? 8 * t + u : 8 * b0 + (u < 4 ? 4 * j + u : 4 * cg + 4 * j + (u - 4));
                val_out[st.v0 + vpos] = s.val;
            }
        }
    }
}

std::vector<u32> row_groups(long long n, const std::function<long long(long long)> &len, long long nnz,
                            long long groups, long long rcap)
{
    std::vector<u32> row0{0};
    const long long target = std::max<long long>(1, (nnz + groups - 1) / groups);
    long long cur = 0;
    for (long long i = 0; i < n; ++i) {
        const long long rows = i - row0.back();
        if (rows > 0 && (rows >= rcap || cur >= target)) {
            row0.push_back((u32)i);
            cur = 0;
        }
        cur += len(i);
    }
    row0.push_back((u32)n);
    return row0;
}

}  // namespace

bool panel_layout(long long n, long long nc, const long long *ptr, const u32 *col, const u32 *val,
                  const unsigned char *cls, u32 m, bool pm_on, int force_q, int nv,
                  const std::function<int(int, bool)> &max_clusters, PanelHost &H)
{
    const std::function<long long(long long)> len = [&](long long i) {
        const long long L = ptr[i + 1] - ptr[i];
        return L > kPanelLong ? 0LL : L;
    };
    long long nnz = 0;
    for (long long i = 0; i < n; ++i) nnz += len(i);
    if (n <= 0 || nc <= 0 || nnz == 0 || nnz >= (1LL << 31) || nc >= (1LL << 31) - 65536) return false;
    const bool small = m <= 65536u;
    const bool tiny = m <= 256u && nv == 1;  // u8 x and values (one vector per pass)
    // odd m in (2^16, 2^31): each value v is stored as v 2^32 mod m, so that
    // the kernel's Montgomery reduction of v' x gives v x mod m (in [0, 2m))
    const bool mont = !small && (m & 1u) != 0 && m < 0x80000000u;
    if (nv != 1 && nv != 2 && !(nv == 4 && small)) return false;
    // bytes of x per column and of row sums per row: nv vectors interleaved
    const int xb = tiny ? 1 : (small ? 2 : 4) * nv, vb = tiny ? 1 : small ? 2 : 4, ab = (small ? 4 : 8) * nv;
    const int ebytes = 4 + vb;
    const int min_sb = 8192 + 1024 * ebytes;
    const long long rcap = std::min<long long>(65536, (kPanelSmemMax - kPanelBarBytes - kPanelDescBytes -
                                                       kPanelStages * min_sb) / ab);

    // column counts, and column groups of q balanced by entries with
    // boundaries on multiples of 64 columns
    std::vector<long long> ccount((size_t)nc, 0);
    for (long long i = 0; i < n; ++i)
        if (len(i))
            for (long long k = ptr[i]; k < ptr[i + 1]; ++k) ccount[col[k]]++;
    auto col_bounds = [&](int cq) {
        std::vector<long long> b{0};
        long long cur = 0;
        for (long long c = 0; c < nc && (int)b.size() < cq; ++c) {
            cur += ccount[c];
            if (cur * cq >= nnz * (long long)b.size() && (c + 1) % 64 == 0 && c + 1 < nc) b.push_back(c + 1);
        }
        while ((int)b.size() < cq) b.push_back(nc);  // empty trailing groups
        b.push_back(nc);
        return b;
    };

    // cluster size (column groups): the fewest waves of clusters, then the
    // most SMs busy, then the larger q; row groups, one per resident
    // cluster, balanced by entries under the shared-memory row cap
    struct Cand {
        int c = 0;
        long long waves = 0, used = 0;
        std::vector<u32> r;
    };
    Cand cand[3];
    int q = 0, nclus = 0;
    long long best_waves = 0, best_used = 0;
    std::vector<u32> row0;
    for (int cq : {1, 2, 4}) {
        if (force_q > 0 && cq != force_q) continue;
        if (force_q <= 0 && cq > 1 && nc < 2LL * cq * 8192) break;
        const int c = max_clusters(cq, small);
        if (c <= 0) continue;
        std::vector<u32> r = row_groups(n, len, nnz, c, rcap);
        const long long G = (long long)r.size() - 1;
        const long long waves = (G + c - 1) / c, used = std::min<long long>(G, c) * cq;
        Cand &k = cand[cq == 1 ? 0 : cq == 2 ? 1 : 2];
        k.c = c;
        k.waves = waves;
        k.used = used;
        k.r = r;
        if (q == 0 || waves < best_waves || (waves == best_waves && used >= best_used)) {
            q = cq;
            nclus = c;
            best_waves = waves;
            best_used = used;
            row0.swap(r);
        }
    }
    if (q == 0) return false;
    if (force_q <= 0 && cand[0].c > 0 && cand[1].c > 0 && cand[0].waves == 1 && cand[1].waves == 1) {
        // One or two CTAs per cluster, both in one wave: two only when the
        // columns are spread over the row groups (each row group's entries
        // split about evenly between the two column groups: local structure
        // such as bands or blocks leaves one CTA of each pair idle) and x
        // outweighs the entries in what a CTA streams (x bytes of all
        // columns at least twice a CTA's entry bytes).  Rule read off
        // whole-plan timings of 1 350 generated matrices; clusters of four
        // rarely won there.
        const std::vector<long long> b2 = col_bounds(2);
        const std::vector<u32> &r2 = cand[1].r;
        long long sum_max = 0;
        for (size_t g = 0; g + 1 < r2.size(); ++g) {
            long long e0 = 0, e1 = 0;
            for (long long i = r2[g]; i < (long long)r2[g + 1]; ++i)
                if (len(i))
                    for (long long k = ptr[i]; k < ptr[i + 1]; ++k) (col[k] < (u32)b2[1] ? e0 : e1)++;
            sum_max += std::max(e0, e1);
        }
        const bool balanced = 2.0 * (double)sum_max <= 1.25 * (double)nnz;
        const double x_over_e = (double)nc * xb * cand[0].c / ((double)nnz * ebytes);
        const int pick = balanced && x_over_e >= 2.0 ? 1 : 0;
        q = pick ? 2 : 1;
        nclus = cand[pick].c;
        row0 = cand[pick].r;
    }
    const long long ng = (long long)row0.size() - 1;
    long long rows_max = 1;
    for (long long g = 0; g < ng; ++g) rows_max = std::max<long long>(rows_max, row0[g + 1] - row0[g]);
    const std::vector<long long> cb = col_bounds(q);
    // stage geometry: px a multiple of 128 bytes, pe a multiple of 64 entries
    long long W = 64;
    for (int j = 0; j < q; ++j) W = std::max<long long>(W, cb[j + 1] - cb[j]);
    const long long acc_bytes = (rows_max * ab + 127) / 128 * 128;
    const long long sb =
        (kPanelSmemMax - kPanelBarBytes - kPanelDescBytes - acc_bytes) / kPanelStages / 128 * 128;  // x slot + entries
    const double dens = (double)nnz / ((double)ng * q) / (double)W;  // entries per column of a CTA
    const long long cstep = 128 / xb;
    long long pcols = (long long)((double)sb / ((double)xb + 1.15 * ebytes * dens));
    pcols = std::min<long long>({pcols, (long long)(kPanelIdxMask + 1), (W + cstep - 1) / cstep * cstep});
    pcols = std::max<long long>(cstep, pcols / cstep * cstep);
    const long long pg = tiny ? 128 : 64;  // pe * ebytes a multiple of 128
    const long long pe = std::min<long long>((sb - pcols * xb) / ebytes / pg * pg, kPanelMaxPe / pg * pg);
    if (pe < pg) return false;
    const long long eb = pe * ebytes;  // a multiple of 128
    const size_t smem = (size_t)(kPanelStages * (pcols * xb + eb) + kPanelBarBytes + kPanelDescBytes + acc_bytes);

    std::vector<long long> pbase(q + 1, 0);  // global panel ids by group
    for (int j = 0; j < q; ++j) pbase[j + 1] = pbase[j] + std::max<long long>(1, (cb[j + 1] - cb[j] + pcols - 1) / pcols);
    const long long npan = pbase[q];
    std::vector<int> cgrp((size_t)nc);
    std::vector<u32> cpan((size_t)nc);
    for (int j = 0; j < q; ++j)
        for (long long c = cb[j]; c < cb[j + 1]; ++c) {
            cgrp[c] = j;
            cpan[c] = (u32)(pbase[j] + (c - cb[j]) / pcols);
        }
    if (ng * npan >= (1LL << 31)) return false;

    // entries bucketed by (row group, panel), rows ascending within a bucket
    std::vector<long long> bstart((size_t)(ng * npan + 1), 0);
    for (long long g = 0; g < ng; ++g)
        for (long long i = row0[g]; i < row0[g + 1]; ++i)
            if (len(i))
                for (long long k = ptr[i]; k < ptr[i + 1]; ++k) bstart[g * npan + cpan[col[k]] + 1]++;
    for (size_t t = 1; t < bstart.size(); ++t) bstart[t] += bstart[t - 1];
    std::vector<SEnt> bent((size_t)nnz);
    std::vector<unsigned char> bpm((size_t)nnz);
    {
        std::vector<long long> pos(bstart.begin(), bstart.end() - 1);
        for (long long g = 0; g < ng; ++g)
            for (long long i = row0[g]; i < row0[g + 1]; ++i) {
                if (!len(i)) continue;
                for (long long k = ptr[i]; k < ptr[i + 1]; ++k) {
                    const long long c = col[k], pan = cpan[c];
                    const long long xoff = cb[cgrp[c]] + (pan - pbase[cgrp[c]]) * pcols;
                    const long long at = pos[g * npan + pan]++;
                    const bool pm = pm_on && cls[k] != 0;
                    const u32 v = mont ? (u32)(((unsigned long long)val[k] << 32) % m) : val[k];
                    bent[at] = SEnt{(u32)(i - row0[g]), (u32)(c - xoff), v, cls[k] == kMinus ? 1u : 0u};
                    bpm[at] = pm ? 1 : 0;
                }
            }
    }

    // stages, CTA by CTA (CTAs laid out in parallel, then concatenated)
    struct CtaOut {
        std::vector<PanelStage> st;
        std::vector<u32> ent, val;
        long long npad = 0, npm = 0;
    };
    const long long nctas = ng * q;
    std::vector<CtaOut> outs((size_t)nctas);
    auto lay_cta = [&](long long cta) {
        const long long g = cta / q;
        const int j = (int)(cta % q);
        CtaOut &o = outs[(size_t)cta];
        std::vector<SEnt> chunk;
        std::vector<unsigned char> chunk_pm;
        const long long np = pbase[j + 1] - pbase[j], rot = g * np / ng;
        u32 loaded = 0;  // panels copied in so far
        for (long long t0 = 0; t0 < np; ++t0) {
            const long long pan = pbase[j] + (t0 + rot) % np;
            const long long b0 = bstart[g * npan + pan], b1 = bstart[g * npan + pan + 1];
            const u32 xoff = (u32)(cb[j] + (pan - pbase[j]) * pcols);
            for (long long k = b0; k < b1; k += pe - 8) {
                const long long e = std::min<long long>(b1, k + pe - 8);
                chunk.assign(bent.begin() + k, bent.begin() + e);
                chunk_pm.assign(bpm.begin() + k, bpm.begin() + e);
                PanelStage st;
                memset(&st, 0, sizeof st);
                st.xoff = xoff;
                // a new panel takes the slot of the panel kPanelStages back,
                // whose stages all ended before the panels in between began
                st.xs = (loaded % kPanelStages) | (k == b0 ? kPanelNewX : 0u);
                lay_stage(chunk, chunk_pm, xb, ab, small, o.ent, o.val, st, o.npad, o.npm);
                o.st.push_back(st);
            }
            if (b1 > b0) ++loaded;
        }
    };
    {
        const int nth = (int)std::max<long long>(1, std::min<long long>(nctas, std::max(1u, std::thread::hardware_concurrency())));
        std::atomic<long long> next(0);
        std::vector<std::thread> pool;
        for (int w = 0; w < nth; ++w)
            pool.emplace_back([&]() {
                for (long long c; (c = next.fetch_add(1)) < nctas;) lay_cta(c);
            });
        for (auto &th : pool) th.join();
    }
    H = PanelHost();
    H.grp_row0 = row0;
    H.stage_ptr.push_back(0);
    H.ent.reserve((size_t)nnz + 16 * (size_t)(ng * npan));
    H.val.reserve((size_t)nnz + 16 * (size_t)(ng * npan));
    for (long long cta = 0; cta < nctas; ++cta) {
        CtaOut &o = outs[(size_t)cta];
        const u32 kb = (u32)H.ent.size(), vbase = (u32)H.val.size();
        if ((unsigned long long)H.ent.size() + o.ent.size() >= (1ull << 32)) return false;
        for (PanelStage st : o.st) {
            st.k0 += kb;
            st.v0 += vbase;
            H.stage.push_back(st);
        }
        H.ent.insert(H.ent.end(), o.ent.begin(), o.ent.end());
        H.val.insert(H.val.end(), o.val.begin(), o.val.end());
        H.npad += o.npad;
        H.npm += o.npm;
        H.stage_ptr.push_back((u32)H.stage.size());
        CtaOut().st.swap(o.st);
        std::vector<u32>().swap(o.ent);
        std::vector<u32>().swap(o.val);
    }
    if (H.ent.size() >= (1ull << 32)) return false;
    // what the kernel's copies and shared-memory reads rely on, checked once
    // here: 16-byte aligned sources and sizes, stages within the buffers,
    // sections within the stage, panels within the staged x copy
    for (const PanelStage &st : H.stage) {
        const bool ok = st.k0 % 8 == 0 && st.v0 % (tiny ? 16 : 8) == 0 && st.nent % 8 == 0 && st.ngen % 8 == 0 &&
                        (!tiny || (size_t)st.v0 + (st.ngen + 15) / 16 * 16 <= H.val.size()) &&
                        st.npg % 8 == 0 && st.npp % 8 == 0 && st.nent <= (u32)pe && st.ngen <= st.nent &&
                        st.npg <= st.ngen && st.npp <= st.nent - st.ngen &&
                        (size_t)st.k0 + st.nent <= H.ent.size() && (size_t)st.v0 + st.ngen <= H.val.size() &&
                        ((size_t)st.xoff * xb) % 16 == 0 && (long long)st.xoff < nc && (st.xs & kPanelSlotMask) < (u32)kPanelStages;
        if (!ok) return false;
    }
    for (u32 w : H.ent)
        if ((long long)(w & kPanelIdxMask) >= pcols) return false;
    if (H.stage.empty()) {
        PanelStage st;
        memset(&st, 0, sizeof st);
        H.stage.push_back(st);
    }
    H.small = small;
    H.tiny = tiny;
    H.mont = mont;
    H.nv = nv;
    H.q = q;
    H.ngroup = (int)ng;
    H.rows_max = (int)rows_max;
    H.resident = nclus;
    H.px = (int)(pcols * xb);
    H.pe = (int)pe;
    H.eb = (int)eb;
    H.smem = smem;
    H.pcols = pcols;
    H.nstage = (long long)H.stage.size();
    return true;
}

}  // namespace ff

using namespace ff;

// Testing aid (see include/ffspmv.h): the host half of the x-panel layout,
// decoded back to (row, column, value) triples.  No device call is made.
extern "C" ffspmv_status ffspmv_panel_decode(int64_t nrows, int64_t ncols, const int64_t *row_ptr,
                                             const int32_t *col, const uint32_t *values, uint32_t m,
                                             int32_t use_pm1, int32_t q, int32_t nv, int32_t clusters, int64_t cap,
                                             int64_t *out_row, int64_t *out_col, uint32_t *out_val,
                                             int64_t *out_n, double *stats)
{
    if (nrows < 0 || ncols < 0 || !row_ptr || m < 2 || (q != 0 && q != 1 && q != 2 && q != 4) ||
        (nv != 1 && nv != 2 && nv != 4) || clusters < 1 || !out_n || cap < 0)
        return FFSPMV_ERR_ARG;
    const long long nnz = row_ptr[nrows];
    std::vector<u32> v((size_t)nnz), c((size_t)nnz);
    std::vector<unsigned char> cls((size_t)nnz);
    for (long long k = 0; k < nnz; ++k) {
        if (col[k] < 0 || col[k] >= ncols) return FFSPMV_ERR_ARG;
        c[k] = (u32)col[k];
        v[k] = values[k] % m;
        cls[k] = v[k] == 1u ? (unsigned char)kPlus : (m > 2u && v[k] == m - 1u) ? (unsigned char)kMinus : 0;
    }
    PanelHost H;
    const bool ok = panel_layout(nrows, ncols, (const long long *)row_ptr, c.data(), v.data(), cls.data(), m,
                                 use_pm1 == 1, q, nv,
                                 [&](int cq, bool) { return q == 0 ? clusters / cq : cq == q ? clusters : 0; }, H);
    if (!ok) return FFSPMV_ERR_UNSUPPORTED;
    const int xb = H.tiny ? 1 : (H.small ? 2 : 4) * nv, ab = (H.small ? 4 : 8) * nv;  // bytes per column / per row
    // values in Montgomery form decode through the inverse of 2^32 mod m
    // (extended Euclid on (2^32 mod m, m); m is odd there, so it exists)
    unsigned long long rinv = 1;
    if (H.mont) {
        long long r0 = (long long)m, r1 = (long long)((1ull << 32) % m), t0 = 0, t1 = 1;
        while (r1 != 0) {
            const long long qt = r0 / r1, r2 = r0 - qt * r1, t2 = t0 - qt * t1;
            r0 = r1; r1 = r2; t0 = t1; t1 = t2;
        }
        rinv = (unsigned long long)((t0 % (long long)m + (long long)m) % (long long)m);
    }
    long long n = 0, lanes = 0, packs = 0, bad_packs = 0;
    double gwf = 0, awf = 0, slots = 0, aslots = 0;
    for (long long cta = 0; cta < (long long)H.ngroup * H.q; ++cta) {
        const long long g = cta / H.q;
        for (u32 s = H.stage_ptr[cta]; s < H.stage_ptr[cta + 1]; ++s) {
            const PanelStage &st = H.stage[s];
            const int nl = (int)st.nent / 8, nlg = (int)st.ngen / 8, lpg = (int)st.npg / 8, lpp = (int)st.npp / 8;
            for (int b0 = 0; b0 < nl; b0 += 32) {
                const int cc = std::min(32, nl - b0), cg = std::min(32, nlg - b0);
                int xw[8][32], rw[8][32];
                int nxw[8] = {0}, nrw[8] = {0};
                long long keys[32];
                for (int t = b0; t < b0 + cc; ++t) {
                    const int j = t - b0;
                    const bool general = t < nlg;
                    const bool pack = general ? t < lpg : t - nlg < lpp;
                    u32 w[8];
                    for (int u = 0; u < 8; ++u) {
                        const int pos = 8 * b0 + (u < 4 ? 4 * j + u : 4 * cc + 4 * j + (u - 4));
                        w[u] = H.ent[st.k0 + pos];
                        u32 value;
                        if (general) {
                            const int vpos = H.small ? 8 * t + u : 8 * b0 + (u < 4 ? 4 * j + u : 4 * cg + 4 * j + (u - 4));
                            value = H.val[st.v0 + vpos];
                            if (H.mont) value = (u32)((unsigned long long)value * rinv % m);
                        } else {
                            value = (w[u] & kPanelNeg) ? m - 1u : 1u;
                        }
                        const u32 idx = w[u] & kPanelIdxMask;
                        xw[u][nxw[u]++] = (int)(xb == 1 ? idx >> 2 : xb == 2 ? idx >> 1 : idx * (u32)(xb / 4));  // first 4-byte word
                        if (!pack) rw[u][nrw[u]++] = (int)(w[u] >> 16);
                        if (value == 0) continue;  // padding
                        if (n < cap) {
                            out_row[n] = (int64_t)H.grp_row0[g] + (w[u] >> 16);
                            out_col[n] = (int64_t)st.xoff + idx;
                            out_val[n] = value;
                        }
                        ++n;
                    }
                    if (pack) {
                        for (int u = 1; u < 8; ++u)
                            if ((w[u] >> 16) != (w[0] >> 16)) ++bad_packs;  // not one row
                        ++packs;
                    }
                    // the kernel's segmented-sum key: a row per section, unique otherwise
                    keys[j] = pack ? (long long)((w[0] >> 16) | (general ? 0u : 0x20000u)) : -1 - j;
                    ++lanes;
                }
                // the lanes of one key must be contiguous within the warp
                for (int a = 0; a < cc; ++a)
                    for (int b = a + 2; b < cc; ++b)
                        if (keys[b] == keys[a] && keys[b - 1] != keys[a]) ++bad_packs;
                // wavefronts: distinct words per bank (gathers), lanes per bank (atomics)
                for (int u = 0; u < 8; ++u) {
                    int bankw[32] = {0};
                    std::vector<int> seen(xw[u], xw[u] + nxw[u]);
                    std::sort(seen.begin(), seen.end());
                    seen.erase(std::unique(seen.begin(), seen.end()), seen.end());
                    for (int wd : seen) bankw[wd & 31]++;
                    gwf += *std::max_element(bankw, bankw + 32);
                    slots += 1;
                    if (nrw[u]) {
                        int bankr[32] = {0};
                        for (int k = 0; k < nrw[u]; ++k) bankr[rbank_of((u32)rw[u][k], ab)]++;
                        awf += *std::max_element(bankr, bankr + 32);
                        aslots += 1;
                    }
                }
            }
        }
    }
    *out_n = n;
    if (stats) {
        stats[0] = (double)H.nstage;
        stats[1] = lanes ? (double)packs / (double)lanes : 0.0;
        stats[2] = slots ? gwf / slots : 0.0;
        stats[3] = aslots ? awf / aslots : 0.0;
        stats[4] = (double)H.npm;
        stats[5] = (double)H.npad;
        stats[6] = (double)H.px;
        stats[7] = (double)H.pe;
        stats[8] = (double)bad_packs;
        stats[9] = (double)H.q;
    }
    return FFSPMV_OK;
}
