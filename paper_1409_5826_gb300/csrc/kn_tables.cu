// kn_tables.cu -- a network's host-side set-up and its device tables:
// validation, the sorted and bank-aware reaction order, the reactant table,
// and the sliced gather list with its bank-aware term order and self-check.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>

#include "kn_host.h"

namespace kn {
namespace {
// Bank-aware order of one slice's terms.  Step k of a slice loads
// V[idx(k, l)] for the warp's 32 lanes l; the load takes one shared-memory
// wavefront when the words lie in distinct banks -- the index mod 32 for
// 4-byte values; 8-byte values take a bank pair (index mod 16), two lanes per
// pair in one step -- or are the same word.  A lane may sum its piece in any
// order, so each step is a maximum matching of lanes to banks (augmenting
// paths, Kuhn's method): lanes that must take a term now to end within the
// slice length come first, then the others by remaining terms; a lane that
// must take a term and is not matched takes one anyway (a conflict), an
// unmatched optional lane reads the zero entry (all such reads are one word).
// Returns the slice length (grows only when a lane could not keep up).
static int schedule_slice(const std::vector<std::vector<uint16_t>>& in, int len, int nbank, int cap, uint16_t zero,
                          std::vector<std::vector<uint16_t>>& out) {
    const int NL = (int)in.size();
    std::vector<std::vector<uint16_t>> rem = in;
    out.assign(NL, {});
    const int zb = zero % nbank;
    for (int k = 0;; ++k) {
        int mx = 0, busy = 0;
        for (auto& r : rem) {
            mx = std::max(mx, (int)r.size());
            busy += !r.empty();
        }
        if (mx == 0) return k;
        const int target = std::max(len, k + mx);
        std::vector<int> order;
        for (int l = 0; l < NL; ++l)
            if (!rem[l].empty()) order.push_back(l);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const bool mx_ = (int)rem[x].size() >= target - k, my_ = (int)rem[y].size() >= target - k;
            if (mx_ != my_) return mx_;
            return rem[x].size() > rem[y].size();
        });
        // bank slots: cap each; one slot of the zero bank is kept for padding
        // lanes whenever some lane will pad
        std::vector<int> cap_left(nbank, cap);
        if (busy < NL && cap_left[zb] > 0) cap_left[zb] -= 1;
        std::vector<std::vector<int>> holder(nbank);  // lanes matched to each bank
        std::vector<int> match(NL, -1);
        std::function<bool(int, std::vector<char>&)> augment = [&](int l, std::vector<char>& seen) -> bool {
            for (uint16_t v : rem[l]) {
                const int b = v % nbank;
                if (seen[b]) continue;
                seen[b] = 1;
                if ((int)holder[b].size() < cap_left[b]) {
                    holder[b].push_back(l);
                    match[l] = b;
                    return true;
                }
                for (size_t h = 0; h < holder[b].size(); ++h) {
                    const int o = holder[b][h];
                    if (augment(o, seen)) {  // o moved to another bank
                        holder[b][h] = l;
                        match[l] = b;
                        return true;
                    }
                }
            }
            return false;
        };
        for (int l : order) {
            std::vector<char> seen(nbank, 0);
            augment(l, seen);
        }
        for (int l = 0; l < NL; ++l) {
            uint16_t v = zero;
            if (!rem[l].empty()) {
                int pick = -1;
                if (match[l] >= 0) {
                    for (size_t t = 0; t < rem[l].size(); ++t)
                        if (rem[l][t] % nbank == match[l]) {
                            pick = (int)t;
                            break;
                        }
                } else if ((int)rem[l].size() >= target - k) {
                    pick = 0;  // must keep up: a conflict
                }
                if (pick >= 0) {
                    v = rem[l][pick];
                    rem[l].erase(rem[l].begin() + pick);
                }
            }
            out[l].push_back(v);
        }
    }
}

// The tables of one network for (precision, threads per zone group Q), built
// and checked on the host; `blob` is what goes to the device.
}  // namespace

kn_status build_tables_host(const kn_network* n, int prec, int Q, std::vector<unsigned char>& blob,
                                   Tables& T) {
    const int N = n->N, R = n->R;
    const int zero_idx = R + n->S_r;
    // sorted order: position jn holds caller reaction perm[jn]; reactant slots
    // are numbered in sorted order too
    // reactant-slot partials in planes: partial q of reaction jn at
    // plane_base(q) + jn, plane q holding the reactions with more than q
    // reactants (V = [fluxes R | plane 0: R | plane 1: R - R1 | plane 2: R - R12 | 0])
    const int R1 = n->R1, R12 = n->R12;
    const int plane_base[3] = {R, 2 * R - R1, 3 * R - R1 - R12};
    // rows 0..N-1: F+_i (value index jn, once per product slot naming i);
    // rows N..2N-1: k_i (value index R + reactant slot id naming i)
    std::vector<std::vector<uint16_t>> rows(2 * N);
    for (int jn = 0; jn < R; ++jn) {
        const int j = n->perm[jn];
        for (int q = 0; q < 3; ++q) {
            const int p = n->prod[j * 3 + q];
            if (p >= 0) rows[p].push_back((uint16_t)jn);
        }
        for (int q = 0; q < n->nr[j]; ++q) rows[N + n->reac[j * 3 + q]].push_back((uint16_t)(plane_base[q] + jn));
    }
    for (int r = 0; r < 2 * N; ++r)
        if (rows[r].empty()) rows[r].push_back((uint16_t)zero_idx);  // row written as 0
    const int real_bytes = prec == kPrecFP64 ? 8 : 4;
    const int fspan = fk_span(N, real_bytes);
    const int G = Q, W = G / 32;
    const int spare = fspan;  // padding lanes store here
    // Fk holds (F+_i, k_i) pairs: row r < N (F+) at slot 2r, row N + i (k) at 2i + 1
    auto slot_of = [N](int r) { return r < N ? 2 * r : 2 * (r - N) + 1; };
    auto row_of = [N](int slot) { return slot % 2 ? N + slot / 2 : slot / 2; };
    if ((spare + 1) * real_bytes > 0xffff) return fail(KN_ERR_INVALID_ARG, "network too large for the gather tables");
    size_t maxlen = 0;
    for (auto& r : rows) maxlen = std::max(maxlen, r.size());
    // One layout for a piece cap L.  A row of more than L terms is cut into
    // k = ceil(len / L) pieces placed in k consecutive lanes of one slice
    // (k <= 32), whose sums a segmented warp reduction combines.  Units
    // (rows) in order of piece length fill slices: a slice opens with the
    // longest remaining unit and takes every later unit that still fits its
    // lanes.  Slices go longest-first to the least-loaded warp; the cost is
    // the longest warp's load, a term counting 1 and the segmented reduction
    // of a slice with split rows kSegCost (its five shuffle rounds take about
    // as many instructions as that many terms).
    struct Piece {
        int row, start, len, dst;
    };
    struct Unit {
        int row, k, plen;
    };
    struct Layout {
        std::vector<std::vector<Piece>> slices;  // 32 pieces each
        std::vector<char> seg;                   // the slice holds a split row
        std::vector<std::vector<int>> warp_slices;
        std::vector<int> slice_len;
        int cost = 1 << 30, warp_len = 0, n_split = 0;
    };
    auto layout_for = [&](int L, Layout& out) -> bool {
        Layout lo;
        std::vector<Unit> units;
        for (int r = 0; r < 2 * N; ++r) {
            const int len = (int)rows[r].size();
            const int k = (len + L - 1) / L;
            if (k > 32) return false;
            units.push_back({r, k, (len + k - 1) / k});
            lo.n_split += k > 1;
        }
        std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.plen > y.plen; });
        std::vector<char> taken(units.size(), 0);
        size_t first = 0;
        for (;;) {
            while (first < units.size() && taken[first]) ++first;
            if (first == units.size()) break;
            std::vector<Piece> sl;
            char seg = 0;
            for (size_t u = first; u < units.size() && sl.size() < 32; ++u) {
                if (taken[u] || (int)sl.size() + units[u].k > 32) continue;
                taken[u] = 1;
                const int r = units[u].row, len = (int)rows[r].size(), k = units[u].k;
                seg |= k > 1;
                for (int q = 0, st = 0; q < k; ++q) {
                    const int pl = len / k + (q < len % k ? 1 : 0);
                    sl.push_back({r, st, pl, slot_of(r) * real_bytes});
                    st += pl;
                }
            }
            while (sl.size() < 32) sl.push_back({-1, 0, 0, spare * real_bytes});
            int sl_len = 0;
            for (auto& pc : sl) sl_len = std::max(sl_len, pc.len);
            lo.slice_len.push_back(sl_len);
            lo.seg.push_back(seg);
            lo.slices.push_back(std::move(sl));
        }
        constexpr int kSegCost = 6;
        const int ns = (int)lo.slices.size();
        std::vector<int> order(ns), cost(ns);
        for (int s = 0; s < ns; ++s) {
            order[s] = s;
            cost[s] = lo.slice_len[s] + (lo.seg[s] ? kSegCost : 0);
        }
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
        lo.warp_slices.assign(W, {});
        std::vector<int> load(W, 0), terms(W, 0);
        for (int s : order) {
            const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            lo.warp_slices[w].push_back(s);
            load[w] += cost[s];
            terms[w] += lo.slice_len[s];
        }
        lo.warp_len = *std::max_element(terms.begin(), terms.end());
        lo.cost = *std::max_element(load.begin(), load.end());
        out = std::move(lo);
        return true;
    };
    Layout best;
    int L_best = 0;
    for (int L = 1; L <= (int)maxlen; ++L) {
        Layout lo;
        if (!layout_for(L, lo)) continue;
        if (lo.cost < best.cost || (lo.cost == best.cost && lo.n_split < best.n_split)) {
            best = std::move(lo);
            L_best = L;
        }
    }
    if (!L_best) return fail(KN_ERR_INVALID_ARG, "no gather layout fits %d threads per zone", G);
    // flatten: slices in warp order; header (base into sidx, length | split flag << 31)
    std::vector<uint16_t> wsl(W + 1, 0), sdst, sidx;
    // the terms as byte offsets into V when they fit 16 bits (the loads then
    // need no scaling), else as indices
    const bool byte_off = (zero_idx + 1) * real_bytes <= 0x10000;
    const int vscale = byte_off ? real_bytes : 1;
    std::vector<uint32_t> shdr;
    int n_slices = 0;
    for (int w = 0; w < W; ++w) {
        wsl[w] = (uint16_t)n_slices;
        for (int s : best.warp_slices[w]) {
            std::vector<std::vector<uint16_t>> lanes(32), ordered;
            for (int l = 0; l < 32; ++l) {
                const Piece& pc = best.slices[s][l];
                sdst.push_back((uint16_t)pc.dst);
                for (int k = 0; k < pc.len; ++k) lanes[l].push_back(rows[pc.row][pc.start + k]);
            }
            const int len = schedule_slice(lanes, best.slice_len[s], real_bytes == 4 ? 32 : 16,
                                           real_bytes == 4 ? 1 : 2, (uint16_t)zero_idx, ordered);
            shdr.push_back((uint32_t)sidx.size());
            shdr.push_back((uint32_t)len | (best.seg[s] ? 0x80000000u : 0u));
            const size_t base = sidx.size();
            sidx.resize(base + 32 * (size_t)len, (uint16_t)(zero_idx * vscale));
            for (int l = 0; l < 32; ++l)
                for (int k = 0; k < len; ++k) sidx[base + 32 * (size_t)k + l] = (uint16_t)(ordered[l][k] * vscale);
            ++n_slices;
        }
    }
    wsl[W] = (uint16_t)n_slices;
    // Host check of the tables before they reach a device: every index in
    // range, a split row's pieces in consecutive lanes of a flagged slice, and
    // the gather, run on the host with V[v] = v + 1, giving every row's sum
    // exactly once (integer sums, exact in FP64).
    {
        std::vector<double> got(2 * N, -1.0);
        for (int w = 0; w < W; ++w)
            for (int sl = wsl[w]; sl < wsl[w + 1]; ++sl) {
                const uint32_t base = shdr[2 * sl], len = shdr[2 * sl + 1] & 0x7fffffffu;
                const bool seg = (shdr[2 * sl + 1] >> 31) != 0;
                if (base + 32 * (size_t)len > sidx.size()) return fail(KN_ERR_INTERNAL, "gather table: slice out of range");
                double acc[32];
                for (int l = 0; l < 32; ++l) {
                    acc[l] = 0.0;
                    for (uint32_t k = 0; k < len; ++k) {
                        const int raw = sidx[base + 32 * k + l];
                        if (raw % vscale) return fail(KN_ERR_INTERNAL, "gather table: misaligned value offset");
                        const int v = raw / vscale;
                        if (v > zero_idx) return fail(KN_ERR_INTERNAL, "gather table: value index out of range");
                        acc[l] += v == zero_idx ? 0.0 : (double)v + 1.0;
                    }
                }
                for (int l = 0; l < 32;) {
                    const uint16_t d = sdst[32 * sl + l];
                    int e = l + 1;
                    double sum = acc[l];
                    while (e < 32 && sdst[32 * sl + e] == d) sum += acc[e++];
                    if (d % real_bytes || d / real_bytes > spare) return fail(KN_ERR_INTERNAL, "gather table: bad destination");
                    const int r = d / real_bytes < 2 * N ? row_of(d / real_bytes) : 2 * N;
                    if (r < 2 * N) {
                        if (e - l > 1 && !seg) return fail(KN_ERR_INTERNAL, "gather table: split row in an unflagged slice");
                        if (got[r] >= 0.0) return fail(KN_ERR_INTERNAL, "gather table: row %d stored twice", r);
                        got[r] = sum;
                    }
                    l = e;
                }
            }
        for (int r = 0; r < 2 * N; ++r) {
            double want = 0.0;
            for (uint16_t v : rows[r]) want += v == zero_idx ? 0.0 : (double)v + 1.0;
            if (got[r] != want) return fail(KN_ERR_INTERNAL, "gather table: row %d sums to %g, not %g", r, got[r], want);
        }
    }
    const int real = prec == kPrecFP64 ? 8 : 4;
    const int a_bytes = prec == kPrecMixed ? 4 : 8;  // A is read by the update: FP64 where the update is
    TableLayout tl{};
    int off = 0;
    tl.off_A = off;
    off = pad16(off + a_bytes * N);
    tl.off_rspec = off;
    off = pad16(off + 4 * R);
    tl.off_cexp = off;
    off = pad16(off + real * R);
    tl.off_wsl = off;
    off = pad16(off + 2 * (W + 1));
    tl.off_shdr = off;
    off = pad16(off + 4 * (int)shdr.size());
    tl.off_sdst = off;
    off = pad16(off + 2 * (int)sdst.size());
    tl.off_sidx = off;
    off = pad16(off + 2 * (int)sidx.size());
    tl.bytes = off;
    blob.assign(off, 0);
    for (int i = 0; i < N; ++i) {
        if (a_bytes == 8) {
            memcpy(blob.data() + tl.off_A + 8 * i, &n->A[i], 8);
        } else {
            const float af = (float)n->A[i];
            memcpy(blob.data() + tl.off_A + 4 * i, &af, 4);
        }
    }
    for (int jn = 0; jn < R; ++jn) {
        const int j = n->perm[jn];
        const uint32_t ra = (uint32_t)n->reac[j * 3];
        const uint32_t rb = (uint32_t)(n->nr[j] >= 2 ? n->reac[j * 3 + 1] : N);
        const uint32_t rc = (uint32_t)(n->nr[j] >= 3 ? n->reac[j * 3 + 2] : N);
        const uint32_t rs = ra | rb << 10 | rc << 20;
        memcpy(blob.data() + tl.off_rspec + 4 * jn, &rs, 4);
        const double c = n->tn[j] + 3.0 * (n->nr[j] - 1);
        if (prec == kPrecFP64) {
            memcpy(blob.data() + tl.off_cexp + 8 * jn, &c, 8);
        } else {
            const float cf = (float)c;
            memcpy(blob.data() + tl.off_cexp + 4 * jn, &cf, 4);
        }
    }
    memcpy(blob.data() + tl.off_wsl, wsl.data(), 2 * wsl.size());
    memcpy(blob.data() + tl.off_shdr, shdr.data(), 4 * shdr.size());
    memcpy(blob.data() + tl.off_sdst, sdst.data(), 2 * sdst.size());
    memcpy(blob.data() + tl.off_sidx, sidx.data(), 2 * sidx.size());
    tl.sidx_bytes = byte_off ? 1 : 0;
    T.tl = tl;
    T.L = L_best;
    T.n_slices = n_slices;
    T.warp_len = best.warp_len;
    return KN_OK;
}


// Validation, the sorted reaction order and the host-side network data; no
// device work.
kn_status network_host_setup(const kn_network_desc* d, std::unique_ptr<kn_network>& n,
                                    std::vector<double>& r0) {
    const int N = d->n_species, R = d->n_reactions;
    if (N < 1 || N > kMaxSpecies) return fail(KN_ERR_INVALID_ARG, "n_species %d outside [1, %d]", N, kMaxSpecies);
    if (R < 1 || R > 16383) return fail(KN_ERR_INVALID_ARG, "n_reactions %d outside [1, 16383]", R);
    if (!d->A || !d->reac || !d->prod || !d->ln_k0 || !d->t9_exp)
        return fail(KN_ERR_INVALID_ARG, "kn_network_desc has a NULL array");
    n.reset(new kn_network());
    n->N = N;
    n->R = R;
    n->A.assign(d->A, d->A + N);
    for (int i = 0; i < N; ++i)
        if (!(std::isfinite(n->A[i]) && n->A[i] > 0)) return fail(KN_ERR_INVALID_ARG, "A[%d] must be finite and > 0", i);
    n->reac.assign(d->reac, d->reac + 3 * R);
    n->prod.assign(d->prod, d->prod + 3 * R);
    n->lnk0.assign(d->ln_k0, d->ln_k0 + R);
    n->tn.assign(d->t9_exp, d->t9_exp + R);
    n->nr.resize(R);
    n->slot0.resize(R);
    int slots = 0, pslots = 0;
    double nsum = 0, rsum = 0;
    for (int j = 0; j < R; ++j) {
        if (!std::isfinite(n->lnk0[j]) || !std::isfinite(n->tn[j]))
            return fail(KN_ERR_INVALID_ARG, "reaction %d: non-finite rate parameter", j);
        int c = 0, end = 0;
        for (int q = 0; q < 3; ++q) {
            const int s = n->reac[j * 3 + q];
            if (s < 0) {
                end = 1;
                continue;
            }
            if (end || s >= N) return fail(KN_ERR_INVALID_ARG, "reaction %d: bad reactant list", j);
            ++c;
        }
        if (c == 0) return fail(KN_ERR_INVALID_ARG, "reaction %d has no reactant", j);
        int pc = 0;
        for (int q = 0; q < 3; ++q) {
            const int s = n->prod[j * 3 + q];
            if (s >= N) return fail(KN_ERR_INVALID_ARG, "reaction %d: product id out of range", j);
            if (s >= 0) ++pc;
        }
        if (pc == 0) return fail(KN_ERR_INVALID_ARG, "reaction %d has no product", j);
        n->nr[j] = c;
        n->slot0[j] = slots;
        slots += c;
        pslots += pc;
        nsum += n->tn[j];
        rsum += c - 1;
    }
    n->S_r = slots;
    n->S_p = pslots;
    // sort reactions by reactant count (stable): 1-body, then 2-body, then 3-body
    n->perm.resize(R);
    for (int j = 0; j < R; ++j) n->perm[j] = j;
    std::stable_sort(n->perm.begin(), n->perm.end(), [&](int a, int b) { return n->nr[a] < n->nr[b]; });
    n->R1 = n->R12 = 0;
    for (int j = 0; j < R; ++j) {
        n->R1 += n->nr[j] == 1;
        n->R12 += n->nr[j] <= 2;
    }
    // Within each class, a warp of the flux pass handles an aligned block of
    // 32 consecutive sorted reactions and loads reactant q's abundance for
    // each; the loads are one wavefront when the species lie in distinct
    // banks (species mod 32) or coincide.  Greedy order: each position of a
    // block takes the remaining reaction of its class that adds the fewest
    // bank conflicts with what the block already reads, per operand.
    {
        const int bounds[4] = {0, n->R1, n->R12, R};
        std::vector<int> sorted(n->perm);
        for (int cls = 0; cls < 3; ++cls) {
            std::vector<int> pool(sorted.begin() + bounds[cls], sorted.begin() + bounds[cls + 1]);
            std::vector<char> used(pool.size(), 0);
            int block = -1;
            // distinct species the block reads per (operand, bank)
            std::vector<std::vector<std::vector<int>>> words(3, std::vector<std::vector<int>>(32));
            for (int pos = bounds[cls]; pos < bounds[cls + 1]; ++pos) {
                if (pos / 32 != block) {
                    block = pos / 32;
                    for (auto& wq : words)
                        for (auto& wb : wq) wb.clear();
                }
                int best = -1, best_cost = 1 << 30;
                for (size_t c = 0; c < pool.size() && best_cost > 0; ++c) {
                    if (used[c]) continue;
                    const int j = pool[c];
                    int cost = 0;
                    for (int q = 0; q < n->nr[j]; ++q) {
                        const int sp = n->reac[j * 3 + q];
                        const auto& wb = words[q][sp % 32];
                        cost += !wb.empty() && std::find(wb.begin(), wb.end(), sp) == wb.end();
                    }
                    if (cost < best_cost) {
                        best_cost = cost;
                        best = (int)c;
                    }
                }
                used[best] = 1;
                const int j = pool[best];
                n->perm[pos] = j;
                for (int q = 0; q < n->nr[j]; ++q) {
                    const int sp = n->reac[j * 3 + q];
                    auto& wb = words[q][sp % 32];
                    if (std::find(wb.begin(), wb.end(), sp) == wb.end()) wb.push_back(sp);
                }
            }
        }
    }
    r0.assign(2 * (size_t)R, 0.0);
    for (int jn = 0; jn < R; ++jn) {
        const int j = n->perm[jn];
        r0[2 * jn] = n->lnk0[j];
        r0[2 * jn + 1] = n->tn[j];
        n->cmax = std::max(n->cmax, std::fabs(n->tn[j] + 3.0 * (n->nr[j] - 1)));
    }
    if (R + slots + 1 > 0xffff) return fail(KN_ERR_INVALID_ARG, "network too large for 16-bit gather indices");
    n->nbar = nsum / R;
    n->rbar = rsum / R;
    return KN_OK;
}

}  // namespace kn
