// Host-side choice of the on-chip samplers' slot order and of each spin's neighbour order, made
// against shared-memory bank conflicts in the neighbour gathers of the force (the coupling sums
// of Eq. 4 and 6).
//
// In the sparse samplers, thread t of a block of n * Rb threads holds spin slot_spin[t / Rb] for
// replica lane t % Rb and, in gather round d, reads the phi word spin_slot[c] * Rb + t % Rb of its
// d-th neighbour c in CSR order (its own word past its degree). Shared memory serves a warp's
// 4-byte reads in one pass when their words are distinct modulo 32 (the banks), and a warp's
// 8-byte reads in one pass per half-warp when each half's words are distinct modulo 16; a word
// read by several lanes is broadcast, and each further distinct word in one bank costs a pass.
// On random 3-regular graphs of n = 1024 the column order costs 18.4 passes per warp for the
// three 8-byte gathers of a step against 6 without conflicts, which left the FP32 pair sampler
// bound by shared memory (a conflict-free circulant graph of the same size ran 18 % faster).
//
// Two local searches, both from the degree-sorted slot order with neighbours by column, with a
// fixed-seed generator so that the layout is a pure function of the graph:
//  1. slots: exchanges of two spins' slots, judged by the bank loads of every half-warp (8-byte
//     words modulo 16) and warp (4-byte words modulo 32) summed over the rounds. Their sum of
//     squares is least when every bank takes one read per round, the condition under which the
//     rounds can be ordered without a conflict (a D-regular bipartite multigraph of threads and
//     banks splits into D perfect matchings, König). Annealed to zero temperature.
//  2. orders: each visited spin takes the order of its reads (among all orders when the degree
//     is at most 4) that gives the fewest passes, 8-byte passes weighted 4 to 1 over 4-byte ones
//     (the FP32 pair and float16 four-replica forms gather 8 bytes, the single-replica and
//     float16 pair forms 4); the counts are updated read by read, so a try costs O(rounds x Rb).
// Neighbour order changes only the order of the force's FP32 sums; slot order changes nothing.
#pragma once

#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace moq {

// Replicas per block whose warps are fullest among blocks of up to about 256 threads (the
// smaller on ties): the samplers' choice when the replica count does not limit it.
inline int fullest_warp_rb(int n)
{
    const int hi = std::max(1, std::min(32, 256 / n));
    int rb = 1;
    double best = -1.0;
    for (int c = 1; c <= hi; ++c) {
        const int threads = n * c;
        const double util = (double)threads / (32.0 * (double)((threads + 31) / 32));
        if (util > best + 0.01) {
            best = util;
            rb = c;
        }
    }
    return rb;
}

class GatherLayout {
public:
    static constexpr int kMaxDeg = 8;

    // nbr: n rows of kMaxDeg entries, the first deg[i] of row i its neighbours (ascending)
    GatherLayout(int n, int rb, std::vector<int32_t> nbr, std::vector<int32_t> deg)
        : n_(n), rb_(rb), nbr_(std::move(nbr)), deg_(std::move(deg))
    {
        T_ = n_ * rb_;
        D_ = 0;
        for (int i = 0; i < n_; ++i) D_ = std::max(D_, (int)deg_[i]);
        spin_at_.resize(n_);
        for (int i = 0; i < n_; ++i) spin_at_[i] = i;
        std::stable_sort(spin_at_.begin(), spin_at_.end(), [&](int32_t a, int32_t b) { return deg_[a] > deg_[b]; });
        slot_of_.resize(n_);
        for (int s = 0; s < n_; ++s) slot_of_[spin_at_[s]] = s;
        H_ = (T_ + 15) / 16;
        W_ = (T_ + 31) / 32;
        c8_.assign((size_t)H_ * std::max(D_, 1), 0);
        c4_.assign((size_t)W_ * std::max(D_, 1), 0);
        stamp_.assign(std::max(T_, 1), 0u);
        refresh();
    }

    int64_t passes8() const { return sum(c8_); }
    int64_t passes4() const { return sum(c4_); }
    int64_t ideal8() const { return (int64_t)H_ * D_; }
    int64_t ideal4() const { return (int64_t)W_ * D_; }
    const std::vector<int32_t>& slot_spin() const { return spin_at_; }
    const std::vector<int32_t>& neighbours() const { return nbr_; }  // gather order, rows of kMaxDeg

    // take the given slot order and gather rows (a permutation of each row's neighbours)
    void set_layout(const std::vector<int32_t>& slot_spin, const std::vector<int32_t>& rows)
    {
        spin_at_ = slot_spin;
        for (int s = 0; s < n_; ++s) slot_of_[spin_at_[s]] = s;
        nbr_ = rows;
        refresh();
    }

    void balance_slots(int64_t moves, uint64_t seed, double temp)
    {
        if (n_ < 2 || D_ == 0) return;
        l8_.assign((size_t)H_ * 16, 0);
        l4_.assign((size_t)W_ * 32, 0);
        for (int i = 0; i < n_; ++i)
            for (int d = 0; d < D_; ++d) load(i, d, +1);
        uint64_t s = seed;
        std::vector<int32_t> reads;
        for (int64_t m = 0; m < moves; ++m) {
            const uint64_t r = next(s);
            const int u = (int)((r >> 8) % (uint64_t)n_);
            int v = (int)((r >> 36) % (uint64_t)(n_ - 1));
            if (v >= u) ++v;
            reads.clear();
            moving_reads(u, reads);
            moving_reads(v, reads);
            std::sort(reads.begin(), reads.end());
            reads.erase(std::unique(reads.begin(), reads.end()), reads.end());
            int64_t delta = 0;
            for (int32_t q : reads) delta += load(q >> 4, q & 15, -1);
            swap_slots(u, v);
            for (int32_t q : reads) delta += load(q >> 4, q & 15, +1);
            bool keep = delta <= 0;
            const double t = temp * (1.0 - (double)m / (double)moves);
            if (!keep && t > 0.0) keep = (double)(next(s) >> 11) * 0x1.0p-53 < std::exp(-(double)delta / t);
            if (!keep) {
                for (int32_t q : reads) load(q >> 4, q & 15, -1);
                swap_slots(u, v);
                for (int32_t q : reads) load(q >> 4, q & 15, +1);
            }
        }
        refresh();
    }

    // `sweeps` passes over all spins, each taking the order of its reads with the fewest weighted
    // passes (a uniform choice among equal ones, which walks plateaus). The counts are kept per
    // cell and updated read by read (Counts below), so trying an order costs O(rounds x Rb).
    void order_reads(int sweeps, uint64_t seed)
    {
        if (D_ < 1) return;
        Counts cnt(*this);
        uint64_t rs = seed ^ 0x5851F42D4C957F2Dull;
        int hs[4], ws[4];
        for (int sw = 0; sw < sweeps; ++sw) {
            for (int u = 0; u < n_; ++u) {
                const int dg = deg_[u];
                if (dg < 2) continue;
                const int t0 = slot_of_[u] * rb_, t1 = t0 + rb_ - 1;
                int nh = 0, nw = 0;
                for (int h = t0 / 16; h <= t1 / 16; ++h) hs[nh++] = h;
                for (int w = t0 / 32; w <= t1 / 32; ++w) ws[nw++] = w;
                auto cost = [&]() {
                    int64_t c = 0;
                    for (int d = 0; d < dg; ++d) {
                        for (int q = 0; q < nh; ++q) c += 4 * cnt.max8[hs[q] * D_ + d];
                        for (int q = 0; q < nw; ++q) c += cnt.max4[ws[q] * D_ + d];
                    }
                    return c;
                };
                int32_t* row = &nbr_[(size_t)u * kMaxDeg];
                int32_t best[kMaxDeg], cur[kMaxDeg];
                std::copy(row, row + dg, best);
                int64_t best_cost = cost();
                if (dg <= 4) {
                    std::copy(row, row + dg, cur);
                    std::sort(cur, cur + dg);
                    int ties = 0;
                    best_cost = INT64_MAX;
                    do {
                        cnt.set_row(u, cur);
                        const int64_t c = cost();
                        if (c < best_cost) {
                            best_cost = c;
                            ties = 1;
                            std::copy(cur, cur + dg, best);
                        } else if (c == best_cost && next(rs) % (uint64_t)(++ties) == 0) {
                            std::copy(cur, cur + dg, best);
                        }
                    } while (std::next_permutation(cur, cur + dg));
                } else {
                    uint64_t s = seed ^ ((uint64_t)u * 0x9E3779B97F4A7C15ull) ^ (uint64_t)sw;
                    for (int k = 0; k < 24; ++k) {
                        const uint64_t r = next(s);
                        const int a = (int)(r % (uint64_t)dg), b = (int)((r >> 20) % (uint64_t)dg);
                        std::copy(best, best + dg, cur);
                        std::swap(cur[a], cur[b]);
                        cnt.set_row(u, cur);
                        const int64_t c = cost();
                        if (c <= best_cost) {
                            best_cost = c;
                            std::copy(cur, cur + dg, best);
                        }
                    }
                }
                cnt.set_row(u, best);
            }
        }
        refresh();
    }

private:
    // Per cell (half-warp or warp, round) the multiplicity of every word read, the distinct words
    // per bank, how many banks hold each count, and the largest count (the cell's passes).
    struct Counts {
        GatherLayout& L;
        std::vector<uint8_t> mult8, mult4, bank8, bank4;
        std::vector<uint16_t> hist8, hist4;
        std::vector<int> max8, max4;

        explicit Counts(GatherLayout& l) : L(l)
        {
            const size_t c8 = (size_t)L.H_ * L.D_, c4 = (size_t)L.W_ * L.D_;
            mult8.assign(c8 * L.T_, 0);
            mult4.assign(c4 * L.T_, 0);
            bank8.assign(c8 * 16, 0);
            bank4.assign(c4 * 32, 0);
            hist8.assign(c8 * 17, 0);
            hist4.assign(c4 * 33, 0);
            max8.assign(c8, 0);
            max4.assign(c4, 0);
            for (size_t c = 0; c < c8; ++c) hist8[c * 17] = 16;
            for (size_t c = 0; c < c4; ++c) hist4[c * 33] = 32;
            for (int t = 0; t < L.T_; ++t)
                for (int d = 0; d < L.D_; ++d) add(t, d, L.word_of(t, d), +1);
        }

        void add(int t, int d, int word, int sign)
        {
            bump(t >> 4, d, word, sign, 16, mult8, bank8, hist8, max8);
            bump(t >> 5, d, word, sign, 32, mult4, bank4, hist4, max4);
        }

        void bump(int g, int d, int word, int sign, int banks, std::vector<uint8_t>& mult, std::vector<uint8_t>& bank,
                  std::vector<uint16_t>& hist, std::vector<int>& mx)
        {
            const size_t c = (size_t)g * L.D_ + d;
            uint8_t& m = mult[c * L.T_ + word];
            if (sign > 0 ? m++ != 0 : --m != 0) return;  // a word already (still) read: no bank change
            uint8_t& b = bank[c * banks + word % banks];
            uint16_t* h = &hist[c * (banks + 1)];
            --h[b];
            b = (uint8_t)(b + sign);
            ++h[b];
            if (b > mx[c]) mx[c] = b;
            while (mx[c] > 0 && h[mx[c]] == 0) --mx[c];
        }

        // spin u's reads in the given order (rounds below its degree)
        void set_row(int u, const int32_t* order)
        {
            int32_t* row = &L.nbr_[(size_t)u * kMaxDeg];
            for (int d = 0; d < L.deg_[u]; ++d) {
                if (row[d] == order[d]) continue;
                for (int lp = 0; lp < L.rb_; ++lp) {
                    const int t = L.slot_of_[u] * L.rb_ + lp;
                    add(t, d, L.slot_of_[row[d]] * L.rb_ + lp, -1);
                    add(t, d, L.slot_of_[order[d]] * L.rb_ + lp, +1);
                }
                row[d] = order[d];
            }
        }
    };

    // the word thread t reads in round d
    int word_of(int t, int d) const
    {
        const int sl = t / rb_, lp = t - sl * rb_;
        const int i = spin_at_[sl];
        const int c = d < deg_[i] ? nbr_[(size_t)i * kMaxDeg + d] : i;
        return slot_of_[c] * rb_ + lp;
    }

    static int64_t sum(const std::vector<int>& v)
    {
        int64_t c = 0;
        for (int x : v) c += x;
        return c;
    }

    static uint64_t next(uint64_t& s)
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);  // splitmix64
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }

    void refresh()
    {
        for (int h = 0; h < H_; ++h)
            for (int d = 0; d < D_; ++d) c8_[h * D_ + d] = passes(16 * h, 16, d, 16);
        for (int w = 0; w < W_; ++w)
            for (int d = 0; d < D_; ++d) c4_[w * D_ + d] = passes(32 * w, 32, d, 32);
    }

    void swap_slots(int u, int v)
    {
        std::swap(slot_of_[u], slot_of_[v]);
        spin_at_[slot_of_[u]] = u;
        spin_at_[slot_of_[v]] = v;
    }

    // passes of the `len` threads from t0 in round d, words distinct modulo `banks`
    int passes(int t0, int len, int d, int banks)
    {
        int cnt[32] = {0};
        if (++epoch_ == 0) {
            std::fill(stamp_.begin(), stamp_.end(), 0u);
            epoch_ = 1;
        }
        int mx = 0;
        const int t1 = std::min(t0 + len, T_);
        for (int t = t0; t < t1; ++t) {
            const int sl = t / rb_, lp = t - sl * rb_;
            const int i = spin_at_[sl];
            const int c = d < deg_[i] ? nbr_[(size_t)i * kMaxDeg + d] : i;
            const int word = slot_of_[c] * rb_ + lp;
            if (stamp_[word] == epoch_) continue;
            stamp_[word] = epoch_;
            mx = std::max(mx, ++cnt[word % banks]);
        }
        return mx;
    }

    // read (i, d), spin i's round-d read (its d-th neighbour, or itself past its degree):
    // adds `sign` to its bank loads, returns the change of the weighted sum of squared loads
    int64_t load(int i, int d, int sign)
    {
        const int c = d < deg_[i] ? nbr_[(size_t)i * kMaxDeg + d] : i;
        int64_t delta = 0;
        for (int lp = 0; lp < rb_; ++lp) {
            const int t = slot_of_[i] * rb_ + lp, word = slot_of_[c] * rb_ + lp;
            int& a = l8_[(t >> 4) * 16 + (word & 15)];
            int& b = l4_[(t >> 5) * 32 + (word & 31)];
            delta += 4 * (sign > 0 ? 2 * a + 1 : 1 - 2 * a) + (sign > 0 ? 2 * b + 1 : 1 - 2 * b);
            a += sign;
            b += sign;
        }
        return delta;
    }

    // the reads whose thread or word moves with spin x: its own and its neighbours' reads of it
    void moving_reads(int x, std::vector<int32_t>& out) const
    {
        for (int d = 0; d < D_; ++d) out.push_back(x << 4 | d);
        for (int q = 0; q < deg_[x]; ++q) {
            const int c = nbr_[(size_t)x * kMaxDeg + q];
            for (int d = 0; d < deg_[c]; ++d)
                if (nbr_[(size_t)c * kMaxDeg + d] == x) out.push_back(c << 4 | d);
        }
    }

    int n_, rb_, T_ = 0, D_ = 0, H_ = 0, W_ = 0;
    std::vector<int32_t> nbr_, deg_, spin_at_, slot_of_;
    std::vector<int> c8_, c4_, l8_, l4_;
    std::vector<uint32_t> stamp_;
    uint32_t epoch_ = 0;
};

}  // namespace moq

namespace moq {

// One replica per block slot (Rb = 1) on a graph whose spins all have degree D: thread t holds
// slot t, so a read's 8-byte bank is the position (slot mod 16) of the read spin inside its own
// half-warp, and a half-warp's round is conflict-free when its 16 reads hit 16 distinct
// positions. If every position takes exactly D of a half-warp's reads, the reads of that
// half-warp split into D rounds of 16 distinct positions (a D-regular bipartite multigraph of
// spins and positions is the union of D perfect matchings, König), found by alternating paths.
// The slots are chosen by annealing the sum of squared (half-warp, position) loads with two
// moves: exchanging spins of the same position between half-warps (only those two half-warps'
// loads change) and exchanging the positions of two spins of one half-warp (their neighbours'
// half-warps change). Every second move is aimed: it takes a cell above D (kept in a list) and
// moves one of its reads, by sending the reading spin to another half-warp or the read spin to
// another position. Half-warps left with a load above D keep the column order for the local
// order search that follows.
class TransversalPlan {
public:
    static constexpr int kD = GatherLayout::kMaxDeg;

    TransversalPlan(int n, int D, const std::vector<int32_t>& nbr) : n_(n), D_(D), H_((n + 15) / 16), nbr_(nbr)
    {
        slot_of_.resize(n_);
        spin_at_.resize(n_);
        for (int i = 0; i < n_; ++i) slot_of_[i] = spin_at_[i] = i;
        cnt_.assign((size_t)n_ * 16, 0);
        load_.assign((size_t)H_ * 16, 0);
        for (int i = 0; i < n_; ++i)
            for (int q = 0; q < D_; ++q) ++cnt_[(size_t)i * 16 + pos(nbr_[(size_t)i * kD + q])];
        for (int i = 0; i < n_; ++i)
            for (int k = 0; k < 16; ++k) load_[(size_t)half(i) * 16 + k] += cnt_[(size_t)i * 16 + k];
        excess_ = excess();
        at_.assign((size_t)H_ * 16, -1);
        for (int c = 0; c < H_ * 16; ++c)
            if (load_[c] > D_) {
                at_[c] = (int)over_.size();
                over_.push_back(c);
            }
    }

    void anneal(int64_t moves, uint64_t seed, double temp)
    {
        uint64_t s = seed;
        for (int64_t m = 0; m < moves; ++m) {
            const uint64_t r = splitmix(s);
            const double t = temp * (1.0 - (double)m / (double)moves);
            int u = (int)((r >> 8) % (uint64_t)n_);
            if (((r >> 4) & 1) && excess_ > 0) {  // aimed at a cell above D
                const int cell = over_[(size_t)((r >> 40) % (uint64_t)over_.size())];
                const int h = cell >> 4, k = cell & 15;
                // a spin of half h with a neighbour at position k (reservoir pick)
                const int lo = h * 16, cntv = std::min(16, n_ - lo);
                int seen = 0;
                uint64_t z = splitmix(s);
                for (int a = 0; a < cntv; ++a) {
                    const int x = spin_at_[lo + a];
                    if (cnt_[(size_t)x * 16 + k] == 0) continue;
                    if ((z >> 8) % (uint64_t)(++seen) == 0) u = x;
                    z = z * 6364136223846793005ull + 1442695040888963407ull;
                }
                if (seen == 0) continue;
                if ((r & 7) < 4) {  // u to another half-warp, same position
                    const int h2 = (int)((r >> 32) % (uint64_t)H_);
                    const int sv = h2 * 16 + pos(u);
                    if (h2 == h || sv >= n_) continue;
                    const int v = spin_at_[sv];
                    if (keep(halves_delta(u, v), t, s)) swap_halves(u, v);
                } else {  // u's neighbour at position k to another position of its half-warp
                    int c = -1;
                    for (int q = 0; q < D_ && c < 0; ++q)
                        if (pos(nbr_[(size_t)u * kD + q]) == k) c = nbr_[(size_t)u * kD + q];
                    const int hc = half(c), lc = hc * 16, cc = std::min(16, n_ - lc);
                    if (cc < 2) continue;
                    int sv = lc + (int)((r >> 32) % (uint64_t)(cc - 1));
                    if (sv >= slot_of_[c]) ++sv;
                    const int v = spin_at_[sv];
                    const int64_t d = swap_positions(c, v);
                    if (!keep(d, t, s)) swap_positions(c, v);
                }
                continue;
            }
            if ((r & 7) < 5) {  // same position, another half-warp
                const int h2 = (int)((r >> 32) % (uint64_t)H_);
                const int sv = h2 * 16 + pos(u);
                if (h2 == half(u) || sv >= n_) continue;
                const int v = spin_at_[sv];
                if (keep(halves_delta(u, v), t, s)) swap_halves(u, v);
            } else {  // two positions of one half-warp
                const int h = half(u), lo = h * 16, cntv = std::min(16, n_ - lo);
                if (cntv < 2) continue;
                int sv = lo + (int)((r >> 32) % (uint64_t)(cntv - 1));
                if (sv >= slot_of_[u]) ++sv;
                const int v = spin_at_[sv];
                const int64_t d = swap_positions(u, v);
                if (!keep(d, t, s)) swap_positions(u, v);
            }
        }
    }

    // rows (n x kD): each spin's reads in rounds 0..D-1 -- König's split for the half-warps
    // whose positions all take at most D reads, the column order elsewhere; returns how many
    // half-warps were split
    int rounds(std::vector<int32_t>& rows) const
    {
        rows = nbr_;
        int done = 0;
        for (int h = 0; h < H_; ++h) {
            bool ok = true;
            for (int k = 0; k < 16; ++k) ok &= load_[(size_t)h * 16 + k] <= D_;
            if (ok && color_half(h, rows)) ++done;
        }
        return done;
    }

    const std::vector<int32_t>& slot_spin() const { return spin_at_; }

    // reads above D summed over the (half-warp, position) cells
    int64_t excess() const
    {
        int64_t e = 0;
        for (int L : load_) e += std::max(0, L - D_);
        return e;
    }

private:
    static uint64_t splitmix(uint64_t& s)
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    static bool keep(int64_t d, double t, uint64_t& s)
    {
        if (d <= 0) return true;
        if (t <= 0.0) return false;
        return (double)(splitmix(s) >> 11) * 0x1.0p-53 < std::exp(-(double)d / t);
    }
    int pos(int i) const { return slot_of_[i] & 15; }
    int half(int i) const { return slot_of_[i] >> 4; }

    // load (h, k) += sign, returns the change of the sum of squares
    int64_t add(int h, int k, int sign)
    {
        int& L = load_[(size_t)h * 16 + k];
        const int64_t d = sign > 0 ? 2 * L + 1 : 1 - 2 * L;
        excess_ += sign > 0 ? (L >= D_) : -(L > D_);
        L += sign;
        const int cell = h * 16 + k;
        if (L > D_ && at_[cell] < 0) {
            at_[cell] = (int)over_.size();
            over_.push_back(cell);
        } else if (L <= D_ && at_[cell] >= 0) {
            const int last = over_.back();
            over_[at_[cell]] = last;
            at_[last] = at_[cell];
            over_.pop_back();
            at_[cell] = -1;
        }
        return d;
    }

    // the change of the sum of squares that swap_halves(u, v) would make
    int64_t halves_delta(int u, int v) const
    {
        const int* cu = &cnt_[(size_t)u * 16];
        const int* cv = &cnt_[(size_t)v * 16];
        const int* Lu = &load_[(size_t)half(u) * 16];
        const int* Lv = &load_[(size_t)half(v) * 16];
        int64_t d = 0;
        for (int k = 0; k < 16; ++k) {
            const int x = cv[k] - cu[k];
            d += (int64_t)x * (2 * (Lu[k] - Lv[k]) + 2 * x);
        }
        return d;
    }

    int64_t swap_halves(int u, int v)
    {
        const int hu = half(u), hv = half(v);
        int64_t d = 0;
        for (int k = 0; k < 16; ++k) {
            const int a = cnt_[(size_t)u * 16 + k], b = cnt_[(size_t)v * 16 + k];
            for (int q = 0; q < b - a; ++q) d += add(hu, k, +1) + add(hv, k, -1);
            for (int q = 0; q < a - b; ++q) d += add(hu, k, -1) + add(hv, k, +1);
        }
        std::swap(slot_of_[u], slot_of_[v]);
        spin_at_[slot_of_[u]] = u;
        spin_at_[slot_of_[v]] = v;
        return d;
    }

    // spin x leaves position a for b: its neighbours' counts and half-warp loads follow
    int64_t relocate(int x, int a, int b)
    {
        int64_t d = 0;
        for (int q = 0; q < D_; ++q) {
            const int c = nbr_[(size_t)x * kD + q];
            --cnt_[(size_t)c * 16 + a];
            ++cnt_[(size_t)c * 16 + b];
            d += add(half(c), a, -1) + add(half(c), b, +1);
        }
        return d;
    }

    int64_t swap_positions(int u, int v)
    {
        const int pu = pos(u), pv = pos(v);
        int64_t d = relocate(u, pu, pv) + relocate(v, pv, pu);
        std::swap(slot_of_[u], slot_of_[v]);
        spin_at_[slot_of_[u]] = u;
        spin_at_[slot_of_[v]] = v;
        return d;
    }

    // D-edge-colouring of half-warp h's (spin, position) multigraph, colours = rounds
    bool color_half(int h, std::vector<int32_t>& rows) const
    {
        const int lo = h * 16, m = std::min(16, n_ - lo);
        // at[side][node][colour] = edge index or -1; side 0 = spins (0..m-1), 1 = positions
        std::vector<int> at(2 * 16 * D_, -1), col(m * D_, -1), eu(m * D_), ev(m * D_), ec(m * D_);
        auto A = [&](int side, int node, int c) -> int& { return at[((size_t)side * 16 + node) * D_ + c]; };
        for (int a = 0; a < m; ++a) {
            const int i = spin_at_[lo + a];
            for (int q = 0; q < D_; ++q) {
                const int e = a * D_ + q;
                eu[e] = a;
                ev[e] = pos(nbr_[(size_t)i * kD + q]);
                ec[e] = nbr_[(size_t)i * kD + q];
            }
        }
        for (int e = 0; e < m * D_; ++e) {
            const int u = eu[e], v = ev[e];
            int a = -1, b = -1;
            for (int c = 0; c < D_ && a < 0; ++c)
                if (A(0, u, c) < 0) a = c;
            for (int c = 0; c < D_ && b < 0; ++c)
                if (A(1, v, c) < 0) b = c;
            if (a < 0 || b < 0) return false;
            if (A(1, v, a) >= 0) {
                // flip the a/b path from v: alternately a-edges and b-edges, starting with a
                int node = v, side = 1, c1 = a, c2 = b;
                std::vector<int> path;
                for (int f = A(side, node, c1); f >= 0; f = A(side, node, c1)) {
                    path.push_back(f);
                    node = side == 1 ? eu[f] : ev[f];
                    side ^= 1;
                    std::swap(c1, c2);
                }
                for (int f : path) {
                    A(0, eu[f], col[f]) = -1;
                    A(1, ev[f], col[f]) = -1;
                }
                for (int f : path) {
                    col[f] = col[f] == a ? b : a;
                    A(0, eu[f], col[f]) = f;
                    A(1, ev[f], col[f]) = f;
                }
            }
            col[e] = a;
            A(0, u, a) = e;
            A(1, v, a) = e;
        }
        for (int a = 0; a < m; ++a) {
            const int i = spin_at_[lo + a];
            for (int q = 0; q < D_; ++q) rows[(size_t)i * kD + col[a * D_ + q]] = ec[a * D_ + q];
        }
        return true;
    }

    int n_, D_, H_;
    std::vector<int32_t> nbr_, slot_of_, spin_at_;
    std::vector<int> cnt_, load_;
    int64_t excess_ = 0;
    std::vector<int> over_, at_;  // the cells above D, each cell's index there (-1: none)
};

}  // namespace moq

namespace moq {

// The layout for the graph (ei, ej) of n spins, E edges: slot_spin (n, slot -> spin) and remap
// (2E entries): row i's neighbour of rank r by column goes to position remap[rowptr_i + r] of
// the row, rows in spin order with rowptr from the degrees. Returns false, leaving both
// untouched, when the graph is outside the samplers' range (n > 1024, a degree above 8) or
// holds an invalid or repeated edge (the device checks report those). `passes`, if given,
// receives the 8-byte and 4-byte passes of the column layout and of the chosen one.
inline bool plan_gather_layout(int n, int64_t E, const int32_t* ei, const int32_t* ej, std::vector<int32_t>& slot_spin,
                               std::vector<int32_t>& remap, int64_t* passes, int64_t effort)
{
    constexpr int kD = GatherLayout::kMaxDeg;
    if (n < 2 || n > 1024 || E <= 0) return false;
    std::vector<int32_t> deg(n, 0), nbr((size_t)n * kD, 0);
    for (int64_t e = 0; e < E; ++e) {
        const int a = ei[e], b = ej[e];
        if (a < 0 || b < 0 || a >= n || b >= n || a == b) return false;
        if (deg[a] >= kD || deg[b] >= kD) return false;
        nbr[(size_t)a * kD + deg[a]++] = b;
        nbr[(size_t)b * kD + deg[b]++] = a;
    }
    for (int i = 0; i < n; ++i) {
        int32_t* row = &nbr[(size_t)i * kD];
        std::sort(row, row + deg[i]);
        for (int d = 1; d < deg[i]; ++d)
            if (row[d] == row[d - 1]) return false;
    }
    const uint64_t seed = 0x243F6A8885A308D3ull ^ ((uint64_t)n << 32) ^ (uint64_t)E;
    GatherLayout col(n, fullest_warp_rb(n), nbr, deg);
    GatherLayout lay = col;
    // effort: 3n slot exchanges and 3 order sweeps (0.2 ms at n = 42, 3 ms at n = 1024, which is
    // part of every time-to-target clock); 10 sweeps buy 3 of 383 8-byte passes at n = 1024 and
    // 3 of 40 at n = 42 for three times the time
    lay.balance_slots(3LL * n, seed, 0.0);
    lay.order_reads(3, seed + 1);
    const GatherLayout* pick = 4 * lay.passes8() + lay.passes4() <= 4 * col.passes8() + col.passes4() ? &lay : &col;
    // One replica per block slot on a regular graph: effort = m > 0 also runs the transversal
    // plan with m * n exchanges and keeps it where it is better. It is off by default
    // because it costs more than a short job gains: at n = 1024, m = 1000 takes 0.15 s and cuts
    // the 8-byte passes from 382 to 254 (192 without conflicts), about 5 % of an FP32 sampling
    // launch of the two-spin form, 1 % of a float16 one
    int D = 0;
    bool regular = true;
    for (int i = 0; i < n; ++i) D = std::max(D, (int)deg[i]);
    for (int i = 0; i < n; ++i) regular &= deg[i] == D;
    GatherLayout tl = col;
    if (effort > 0 && fullest_warp_rb(n) == 1 && regular && D >= 2) {
        TransversalPlan tp(n, D, nbr);
        tp.anneal(effort * n, seed + 2, 0.0);
        std::vector<int32_t> rows;
        tp.rounds(rows);
        tl.set_layout(tp.slot_spin(), rows);
        tl.order_reads(3, seed + 3);
        if (4 * tl.passes8() + tl.passes4() < 4 * pick->passes8() + pick->passes4()) pick = &tl;
    }
    if (passes) {
        passes[0] = col.passes8();
        passes[1] = col.passes4();
        passes[2] = pick->passes8();
        passes[3] = pick->passes4();
    }
    slot_spin = pick->slot_spin();
    remap.assign((size_t)2 * E, 0);
    const std::vector<int32_t>& order = pick->neighbours();
    int64_t p0 = 0;
    for (int i = 0; i < n; ++i) {
        const int32_t* sorted = &nbr[(size_t)i * kD];
        const int32_t* chosen = &order[(size_t)i * kD];
        for (int r = 0; r < deg[i]; ++r)
            remap[p0 + r] = (int32_t)(std::find(chosen, chosen + deg[i], sorted[r]) - chosen);
        p0 += deg[i];
    }
    return true;
}

}  // namespace moq
