// Host-side gate fusion (paper section IV-D): vertical fusion is the matrix product of gates on
// the same qubits, horizontal fusion the tensor product of gates on disjoint qubits (Eq. 4).
// All products are formed in fp64; each finished fused matrix is rounded to fp32 once.
//
// Greedy rule (the paper fixes only "greedy, at most f qubits"; this is the library's reading):
// gates are scanned in circuit order while a set of open blocks with pairwise disjoint qubit sets
// is kept.  A gate on qubits Q joins the open blocks that touch Q.  If their union with Q has more
// than max_k qubits, the touching blocks with the most qubits outside Q are closed (emitted) until
// the rest fits; the gate then merges with what remains.  Blocks on disjoint qubits commute, so
// emitting a closed block before still-open disjoint blocks keeps the circuit's meaning.
//
// A second pass adds horizontal fusion across the emitted sequence: each emitted block moves back
// over the blocks before it that share no qubit with it (they commute) and merges into the first
// block it meets whose union with it still has at most max_k qubits.
//
// The partition depends only on the gates' qubits, never on matrix values, so the scan records
// how each block's matrix is formed (a small expression: a starting block re-expressed over more
// qubits, then left products by gates and by merged blocks) and the products run afterwards, for
// the chosen partition only, one fused gate per host thread.
#include <algorithm>
#include <array>
#include <future>
#include <memory>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>

#include "sv_internal.h"

namespace svg {

namespace {

// A block's matrix as recorded by the scan: base's matrix (identity when null) re-expressed over
// `qubits`, then left-multiplied by each op in order -- a dense gate over op.gq, or (op.child set)
// another block's matrix over child->qubits.
struct MatNode;
using NodeP = std::shared_ptr<MatNode>;
struct MatOp {
    std::vector<cplx> g;
    std::vector<int> gq;
    NodeP child;
};
struct MatNode {
    std::vector<int> qubits;   // ascending
    NodeP base;
    std::vector<MatOp> ops;
};

NodeP new_node(const std::vector<int> &qubits, NodeP base)
{
    NodeP n = std::make_shared<MatNode>();
    n->qubits = qubits;
    n->base = std::move(base);
    return n;
}

struct Block {
    std::vector<int> qubits;  // ascending
    NodeP node;               // how the matrix is formed (greedy scan)
    std::vector<cplx> mat;    // 2^|qubits| square, local bit j <-> qubits[j] (once evaluated)
    int n_src = 0;
    long long created = 0;
    uint64_t cmask = 0;       // a controlled gate kept whole (qubits = its targets); else 0
    // single-qubit gates absorbed but not yet multiplied in: the block's operator is
    // (product over pend of P_q) * mat; each is folded into the next gate on its qubit, or
    // multiplied in when the block closes (saves a 2^k x 2^k update per single-qubit gate)
    std::vector<std::pair<int, std::array<cplx, 4>>> pend;
};

// Rows r_j = base | off[j] (j < GD) of mat, each `dim` complex entries, replaced by G times them.
// Every column's GD inputs are read before any output of that column is written, so no copy is
// needed, and the column loop runs over contiguous memory.  A complex entry is one two-lane
// vector (GCC's generic vector extension: two doubles per operation on any target); with
// xs = (-Im x, Re x) the product G x is Re G * x + Im G * xs, the same sums in the same order as
// the scalar form.
typedef double v2d __attribute__((vector_size(16)));

template <int GD>
void mix_rows(double *m, size_t dim, size_t base, const size_t *off, const std::vector<cplx> &G)
{
    double gr[GD][GD], gi[GD][GD];
    for (int r = 0; r < GD; ++r)
        for (int j = 0; j < GD; ++j) {
            gr[r][j] = G[(size_t)r * GD + j].real();
            gi[r][j] = G[(size_t)r * GD + j].imag();
        }
    v2d *row[GD];
    for (int j = 0; j < GD; ++j) row[j] = reinterpret_cast<v2d *>(m + 2 * (base | off[j]) * dim);
    for (size_t c = 0; c < dim; ++c) {
        v2d x[GD], xs[GD];
        for (int j = 0; j < GD; ++j) {
            x[j] = row[j][c];
            xs[j] = v2d{-x[j][1], x[j][0]};
        }
        for (int r = 0; r < GD; ++r) {
            v2d y = {0.0, 0.0};
            for (int j = 0; j < GD; ++j) y += gr[r][j] * x[j] + gi[r][j] * xs[j];
            row[r][c] = y;
        }
    }
}

// mat (dim x dim, acting on qubit list T) <- G * mat, where G acts on qubits gq (local bit b of G
// <-> gq[b], every gq[b] in T).  G mixes the rows of mat whose indices differ only in G's bits:
// each such group of rows (visited through its all-zero member) is replaced by G times it.
void left_multiply(std::vector<cplx> &mat, const std::vector<int> &T, const std::vector<cplx> &G,
                   const std::vector<int> &gq)
{
    const int t = (int)T.size();
    const int kg = (int)gq.size();
    const size_t dim = size_t(1) << t;
    const size_t gd = size_t(1) << kg;
    int pos[SV_MAX_K + SV_MAX_CONTROLS];
    size_t gmask = 0;
    for (int b = 0; b < kg; ++b) {
        pos[b] = int(std::find(T.begin(), T.end(), gq[b]) - T.begin());
        gmask |= size_t(1) << pos[b];
    }
    std::vector<size_t> off(gd);
    for (size_t j = 0; j < gd; ++j) {
        size_t o = 0;
        for (int b = 0; b < kg; ++b)
            if ((j >> b) & 1) o |= size_t(1) << pos[b];
        off[j] = o;
    }
    double *m = reinterpret_cast<double *>(mat.data());
    for (size_t base = 0; base < dim; ++base) {
        if (base & gmask) continue;
        switch (kg) {
        case 1: mix_rows<2>(m, dim, base, off.data(), G); break;
        case 2: mix_rows<4>(m, dim, base, off.data(), G); break;
        case 3: mix_rows<8>(m, dim, base, off.data(), G); break;
        case 4: mix_rows<16>(m, dim, base, off.data(), G); break;
        case 5: mix_rows<32>(m, dim, base, off.data(), G); break;
        default: mix_rows<64>(m, dim, base, off.data(), G); break;
        }
    }
}

std::vector<cplx> identity(size_t dim)
{
    std::vector<cplx> m(dim * dim, cplx(0.0, 0.0));
    for (size_t i = 0; i < dim; ++i) m[i * dim + i] = 1.0;
    return m;
}

// M_S (acting on qubit list S) re-expressed on the ascending superset T: M_T = M_S (x) I on T \ S.
std::vector<cplx> expand(const std::vector<cplx> &M, const std::vector<int> &S, const std::vector<int> &T)
{
    const int t = (int)T.size(), sz = (int)S.size();
    if (sz == t) return M;
    const size_t dT = size_t(1) << t, dS = size_t(1) << sz, dR = size_t(1) << (t - sz);
    std::vector<size_t> depS(dS), depR(dR);
    int posS[16], posR[16], nr = 0;
    for (int i = 0; i < sz; ++i) posS[i] = int(std::find(T.begin(), T.end(), S[i]) - T.begin());
    for (int i = 0; i < t; ++i)
        if (std::find(S.begin(), S.end(), T[i]) == S.end()) posR[nr++] = i;
    for (size_t v = 0; v < dS; ++v) {
        size_t o = 0;
        for (int b = 0; b < sz; ++b)
            if ((v >> b) & 1) o |= size_t(1) << posS[b];
        depS[v] = o;
    }
    for (size_t v = 0; v < dR; ++v) {
        size_t o = 0;
        for (int b = 0; b < nr; ++b)
            if ((v >> b) & 1) o |= size_t(1) << posR[b];
        depR[v] = o;
    }
    std::vector<cplx> out(dT * dT, cplx(0.0, 0.0));
    for (size_t e = 0; e < dR; ++e)
        for (size_t r = 0; r < dS; ++r)
            for (size_t c = 0; c < dS; ++c) out[(depS[r] | depR[e]) * dT + (depS[c] | depR[e])] = M[r * dS + c];
    return out;
}

// multiplies every pending single-qubit gate of b into b's matrix (recorded)
void flush_pending(Block &b)
{
    for (auto &pq : b.pend) b.node->ops.push_back(MatOp{std::vector<cplx>(pq.second.begin(), pq.second.end()), {pq.first}, nullptr});
    b.pend.clear();
}

std::vector<cplx> evaluate(const MatNode &n)
{
    std::vector<cplx> M = n.base ? expand(evaluate(*n.base), n.base->qubits, n.qubits) : identity(size_t(1) << n.qubits.size());
    for (const MatOp &op : n.ops) {
        if (op.child) left_multiply(M, n.qubits, evaluate(*op.child), op.child->qubits);
        else left_multiply(M, n.qubits, op.g, op.gq);
    }
    return M;
}

// complex multiply-adds that evaluate(n) performs
double eval_cost(const MatNode &n)
{
    const double d2 = std::ldexp(1.0, 2 * (int)n.qubits.size());
    double c = n.base ? eval_cost(*n.base) + d2 : d2;
    for (const MatOp &op : n.ops)
        c += op.child ? eval_cost(*op.child) + d2 * std::ldexp(1.0, (int)op.child->qubits.size())
                      : d2 * std::ldexp(1.0, (int)op.gq.size());
    return c;
}

// Every block's matrix from its recorded expression; with `parallel`, blocks are shared out to
// host threads, one thread per ~5e5 complex multiply-adds (about half a millisecond: less would
// not pay for starting the thread), else evaluated in order.
void materialize(std::vector<Block> &blocks, bool parallel)
{
    size_t nt = 1;
    if (parallel) {
        double cost = 0.0;
        for (const Block &b : blocks) cost += eval_cost(*b.node);
        nt = (size_t)(cost / 5e5) + 1;
    }
    host_parallel_for(blocks.size(), nt, [&](size_t i) {
        blocks[i].mat = evaluate(*blocks[i].node);
        blocks[i].node.reset();
    });
}

// G (acting on qubit list Q) <- G * P_q for every pending gate of b on a qubit of Q (P applied
// first), and drops those from b.pend
void fold_pending(std::vector<cplx> &G, const std::vector<int> &Q, Block &b)
{
    const size_t d = size_t(1) << Q.size();
    for (size_t i = 0; i < b.pend.size();) {
        const int q = b.pend[i].first;
        const auto it = std::find(Q.begin(), Q.end(), q);
        if (it == Q.end()) { ++i; continue; }
        const size_t bit = size_t(1) << (it - Q.begin());
        const std::array<cplx, 4> &P = b.pend[i].second;
        for (size_t r = 0; r < d; ++r)
            for (size_t c0 = 0; c0 < d; ++c0) {
                if (c0 & bit) continue;
                const size_t c1 = c0 | bit;
                const cplx g0 = G[r * d + c0], g1 = G[r * d + c1];
                G[r * d + c0] = g0 * P[0] + g1 * P[2];
                G[r * d + c1] = g0 * P[1] + g1 * P[3];
            }
        b.pend.erase(b.pend.begin() + (long)i);
    }
}

struct Dense {
    std::vector<int> q;        // qubits: targets then folded controls (local bit order of m)
    std::vector<cplx> m;       // dense matrix with those controls folded in
    uint64_t cmask = 0;        // controls kept as controls (the gate is not fused); else 0
    int src = 1;               // input gates it stands for (0: a factor split off another gate)
};

// A controlled gate as its own block over its ascending targets (the matrix expression only with
// `nodes`).
Block controlled_block(const Dense &d, bool nodes = true)
{
    Block b;
    b.qubits = d.q;
    std::sort(b.qubits.begin(), b.qubits.end());
    if (nodes) {
        b.node = new_node(b.qubits, nullptr);
        b.node->ops.push_back(MatOp{d.m, d.q, nullptr});
    }
    b.n_src = d.src;
    b.cmask = d.cmask;
    return b;
}

constexpr double kMaxTrustedError = 0.25;   // learned mode falls back above this validation error
constexpr int kMaxControlledK = 3;          // targets of a gate kept controlled
constexpr int kMaxStartQubits = 28;         // the small start state of sv_init_apply

// Which touching blocks a gate that does not fit closes first (the greedy rule leaves this open;
// the learned partitioner tries all three): kCloseOutside -- the most qubits outside the gate
// (the library's default), kCloseOldest -- the least recently extended, kCloseLargest -- the most
// qubits.
enum CloseRule : int { kCloseOutside = 0, kCloseOldest = 1, kCloseLargest = 2, kCloseRules = 3 };

// Greedy fusion to at most max_k qubits (larger single gates stay whole), then the horizontal pass.
// With `nodes` false only the partition is planned (qubit sets, no matrix expressions): the
// decisions depend on qubit sets alone, so the plan equals the partition built with nodes.
std::vector<Block> greedy_partition(const std::vector<Dense> &dense, int n_qubits, int max_k, int rule = kCloseOutside,
                                    bool nodes = true)
{
    std::vector<Block> open, emitted;
    long long stamp = 0;
    for (size_t gi = 0; gi < dense.size(); ++gi) {
        const std::vector<int> &Q = dense[gi].q;
        uint64_t qmask = 0;
        for (int q : Q) qmask |= uint64_t(1) << q;
        if (dense[gi].cmask) {
            // a controlled gate is a barrier on every qubit it names: close the blocks it touches
            // (creation order), emit it, keep the others open (disjoint, so they commute with it)
            const uint64_t sm = qmask | dense[gi].cmask;
            std::vector<Block> rest;
            std::vector<Block> closed;
            for (Block &b : open) {
                bool t = false;
                for (int q : b.qubits) t = t || ((sm >> q) & 1);
                (t ? closed : rest).push_back(std::move(b));
            }
            std::sort(closed.begin(), closed.end(), [](const Block &a, const Block &b) { return a.created < b.created; });
            for (Block &b : closed) {
                if (nodes) flush_pending(b);
                emitted.push_back(std::move(b));
            }
            Block cb = controlled_block(dense[gi], nodes);
            cb.created = stamp++;
            emitted.push_back(std::move(cb));
            open.swap(rest);
            continue;
        }
        std::vector<int> touching;
        for (int b = 0; b < (int)open.size(); ++b) {
            for (int q : open[b].qubits)
                if ((qmask >> q) & 1) { touching.push_back(b); break; }
        }
        // close touching blocks with the most qubits outside Q until the union fits
        auto outside = [&](int b) {
            int c = 0;
            for (int q : open[b].qubits) c += !((qmask >> q) & 1);
            return c;
        };
        std::sort(touching.begin(), touching.end(), [&](int a, int b) {
            if (rule == kCloseLargest && open[a].qubits.size() != open[b].qubits.size())
                return open[a].qubits.size() > open[b].qubits.size();
            if (rule == kCloseOutside) {
                const int oa = outside(a), ob = outside(b);
                if (oa != ob) return oa > ob;
            }
            return open[a].created < open[b].created;
        });
        auto union_size = [&](size_t from) {
            uint64_t m = qmask;
            for (size_t i = from; i < touching.size(); ++i)
                for (int q : open[touching[i]].qubits) m |= uint64_t(1) << q;
            return __builtin_popcountll(m);
        };
        size_t first_kept = 0;
        const int limit = std::max(max_k, (int)Q.size());
        while (first_kept < touching.size() && union_size(first_kept) > limit) ++first_kept;
        // emit closed blocks in creation order
        std::vector<int> closed(touching.begin(), touching.begin() + first_kept);
        std::sort(closed.begin(), closed.end(), [&](int a, int b) { return open[a].created < open[b].created; });
        std::vector<int> kept(touching.begin() + first_kept, touching.end());
        std::sort(kept.begin(), kept.end(), [&](int a, int b) { return open[a].created < open[b].created; });
        for (int b : closed) {
            if (nodes) flush_pending(open[b]);
            emitted.push_back(std::move(open[b]));
        }

        // a single-qubit gate on a qubit of one open block stays pending there
        if (Q.size() == 1 && kept.size() == 1 && touching.size() == 1) {
            Block &kb = open[kept[0]];
            if (nodes) {
                const std::vector<cplx> &G = dense[gi].m;
                std::array<cplx, 4> P = {G[0], G[1], G[2], G[3]};
                for (size_t i = 0; i < kb.pend.size(); ++i)
                    if (kb.pend[i].first == Q[0]) {   // G * earlier pending
                        const std::array<cplx, 4> &E = kb.pend[i].second;
                        P = {G[0] * E[0] + G[1] * E[2], G[0] * E[1] + G[1] * E[3], G[2] * E[0] + G[3] * E[2], G[2] * E[1] + G[3] * E[3]};
                        kb.pend.erase(kb.pend.begin() + (long)i);
                        break;
                    }
                kb.pend.push_back({Q[0], P});
            }
            kb.n_src += dense[gi].src;
            kb.created = stamp++;
            continue;
        }

        // merge kept blocks (disjoint, so they commute) and the gate into one block over the union
        uint64_t um = qmask;
        for (int b : kept)
            for (int q : open[b].qubits) um |= uint64_t(1) << q;
        Block nb;
        for (int q = 0; q < n_qubits; ++q)
            if ((um >> q) & 1) nb.qubits.push_back(q);
        nb.n_src = dense[gi].src;
        for (int b : kept)   // pending single-qubit gates carry over (their qubits stay disjoint)
            for (auto &pq : open[b].pend) nb.pend.push_back(pq);
        if (!nodes) {
            for (int b : kept) nb.n_src += open[b].n_src;
        } else if (kept.empty()) {
            nb.node = new_node(nb.qubits, nullptr);
        } else {
            // the first kept block's matrix carries over unchanged when the gate adds no qubit to it
            if (open[kept[0]].qubits == nb.qubits) nb.node = std::move(open[kept[0]].node);
            else nb.node = new_node(nb.qubits, std::move(open[kept[0]].node));
            nb.n_src += open[kept[0]].n_src;
            for (size_t i = 1; i < kept.size(); ++i) {
                nb.node->ops.push_back(MatOp{{}, {}, std::move(open[kept[i]].node)});
                nb.n_src += open[kept[i]].n_src;
            }
        }
        if (nodes) {
            std::vector<cplx> G = dense[gi].m;
            fold_pending(G, Q, nb);   // the pending gates on Q act before this gate
            nb.node->ops.push_back(MatOp{std::move(G), Q, nullptr});
        }
        nb.created = stamp++;
        std::vector<char> drop(open.size(), 0);
        for (int b : touching) drop[b] = 1;
        std::vector<Block> rest;
        rest.reserve(open.size() + 1);
        for (size_t b = 0; b < open.size(); ++b)
            if (!drop[b]) rest.push_back(std::move(open[b]));
        rest.push_back(std::move(nb));
        open.swap(rest);
    }
    std::sort(open.begin(), open.end(), [](const Block &a, const Block &b) { return a.created < b.created; });
    for (Block &b : open) {
        if (nodes) flush_pending(b);
        emitted.push_back(std::move(b));
    }

    // horizontal pass: move each block back over disjoint predecessors and merge where it fits
    std::vector<Block> merged;
    const int kScanBack = 64;
    for (Block &b : emitted) {
        if (b.cmask) {   // controlled gates neither merge nor move
            merged.push_back(std::move(b));
            continue;
        }
        uint64_t bm = 0;
        for (int q : b.qubits) bm |= uint64_t(1) << q;
        const int lim = std::max(max_k, (int)b.qubits.size());
        int target = -1;
        for (int p = (int)merged.size() - 1, steps = 0; p >= 0 && steps < kScanBack; --p, ++steps) {
            uint64_t pm = merged[p].cmask;
            for (int q : merged[p].qubits) pm |= uint64_t(1) << q;
            if (!merged[p].cmask && __builtin_popcountll(pm | bm) <= lim) { target = p; break; }
            if (pm & bm) break;   // cannot move past a block it shares a qubit with
        }
        if (target < 0) {
            merged.push_back(std::move(b));
            continue;
        }
        Block &t = merged[size_t(target)];
        uint64_t um = bm;
        for (int q : t.qubits) um |= uint64_t(1) << q;
        std::vector<int> U;
        for (int q = 0; q < n_qubits; ++q)
            if ((um >> q) & 1) U.push_back(q);
        if (nodes) {
            if (U != t.qubits) t.node = new_node(U, std::move(t.node));   // earlier block first
            t.node->ops.push_back(MatOp{{}, {}, std::move(b.node)});
        }
        t.qubits = std::move(U);
        t.n_src += b.n_src;
    }
    return merged;
}

// Light-cone split for a circuit that starts from a basis state (opts.start_qubits = m): the
// qubit set S grows with each gate's qubits, in circuit order, while it has at most m qubits; a
// gate joins the first part when no earlier gate left out shares a qubit with it (so it commutes
// past all of them) and its qubits lie in S, else its qubits are closed.  The first part is fused
// apart and placed first: a start from a basis state runs it on the small state of S's qubits.
void split_light_cone(const std::vector<Dense> &dense, int m, std::vector<Dense> &first, std::vector<Dense> &rest)
{
    uint64_t S = 0, closed = 0;
    for (const Dense &d : dense) {
        uint64_t q = d.cmask;
        for (int t : d.q) q |= uint64_t(1) << t;
        if (!(q & closed) && __builtin_popcountll(S | q) <= m) {
            S |= q;
            first.push_back(d);
        } else {
            closed |= q;
            rest.push_back(d);
        }
    }
}

// An equivalent gate order for the learned search: each diagonal gate (not kept controlled) moves
// later, to just before the next gate on one of its qubits that is not diagonal (diagonal gates
// commute with each other, and every gate commutes with gates on other qubits); the rest keep their
// order.  Kept controlled gates count as not diagonal.  Returns false when nothing moves.
bool is_diagonal(const Dense &d)
{
    if (d.cmask) return false;
    const size_t D = size_t(1) << d.q.size();
    for (size_t r = 0; r < D; ++r)
        for (size_t c = 0; c < D; ++c)
            if (r != c && std::abs(d.m[r * D + c]) > 1e-12) return false;
    return true;
}

bool defer_diagonals(const std::vector<Dense> &in, std::vector<Dense> &out)
{
    std::vector<char> diag(in.size());
    for (size_t i = 0; i < in.size(); ++i) diag[i] = is_diagonal(in[i]);
    std::vector<size_t> order, pending;
    for (size_t i = 0; i < in.size(); ++i) {
        if (diag[i]) {
            pending.push_back(i);
            continue;
        }
        uint64_t q = in[i].cmask;
        for (int t : in[i].q) q |= uint64_t(1) << t;
        std::vector<size_t> keep;
        for (size_t p : pending) {
            uint64_t pq = 0;
            for (int t : in[p].q) pq |= uint64_t(1) << t;
            if (pq & q) order.push_back(p);
            else keep.push_back(p);
        }
        pending.swap(keep);
        order.push_back(i);
    }
    for (size_t p : pending) order.push_back(p);
    bool moved = false;
    for (size_t i = 0; i < order.size(); ++i) moved = moved || order[i] != i;
    out.clear();
    out.reserve(in.size());
    for (size_t i : order) out.push_back(in[i]);
    return moved;
}

// greedy_partition of the circuit, or of its light-cone part followed by the rest's (*split_at:
// the number of blocks of the first part, 0 without a split)
std::vector<Block> partition(const std::vector<Dense> &dense, const std::vector<Dense> *first, const std::vector<Dense> *rest,
                             int n_qubits, int max_k, int rule = kCloseOutside, size_t *split_at = nullptr, bool nodes = true)
{
    if (split_at) *split_at = 0;
    if (!first) return greedy_partition(dense, n_qubits, max_k, rule, nodes);
    std::vector<Block> a = greedy_partition(*first, n_qubits, max_k, rule, nodes);
    if (split_at) *split_at = a.size();
    std::vector<Block> b = greedy_partition(*rest, n_qubits, max_k, rule, nodes);
    for (Block &x : b) a.push_back(std::move(x));
    return a;
}

uint64_t block_mask(const Block &b)
{
    uint64_t m = b.cmask;
    for (int q : b.qubits) m |= uint64_t(1) << q;
    return m;
}

// Predicted device time of a fused gate by its qubit set and the size of the state it runs on:
// the cheapest kernel path it may take (its CUDA-core path, and its tensor-core path when the
// precision allows one), from the trained model or the caller's cost function.  Predictions are
// kept, so a (qubit set, state size) is scored once.  Keys: the mask with the state size in the top
// bits (masks have at most 34 bits).
uint64_t cost_key(uint64_t mask, int n) { return mask | ((uint64_t)n << 56); }
constexpr uint64_t kPostKey = uint64_t(1) << 55;   // key flag: the gate carries post-phases

class GateCost {
public:
    explicit GateCost(const sv_fuse_opts &o) : o_(o) {}

    // scores every key not scored yet (one batched model call)
    int ensure(const std::vector<uint64_t> &keys)
    {
        std::vector<uint64_t> todo;
        for (uint64_t key : keys)
            if (!known_.count(key)) {
                known_[key] = {0.0, SV_PATH_AUTO};
                todo.push_back(key);
            }
        if (todo.empty()) return SV_OK;
        std::vector<float> X;
        std::vector<std::pair<size_t, int>> rows;   // (index into todo, path)
        std::vector<std::array<int, SV_MAX_K>> tg(todo.size());
        for (size_t t = 0; t < todo.size(); ++t) {
            const int n = (int)(todo[t] >> 56);
            const bool post = (todo[t] & kPostKey) != 0;
            FusedGate g;
            for (int q = 0; q < 55; ++q)
                if ((todo[t] >> q) & 1) g.targets[g.k++] = q;
            std::copy(g.targets, g.targets + SV_MAX_K, tg[t].begin());
            const int tc = o_.precision == SV_PREC_TF32 ? SV_PATH_TC_TF32 : SV_PATH_TC_BF16X3;
            std::vector<int> paths;
            if (post) {   // only the tensor-core kernel applies post-phases
                paths.push_back(tc);
            } else {
                paths.push_back(classify_path(g, n, SV_PREC_FP32, SV_MAX_K + 1, SV_PATH_AUTO));
                if (o_.precision != SV_PREC_FP32 && g.k >= 4 && n >= g.k + 5) paths.push_back(tc);
            }
            for (int p : paths) {
                rows.push_back({t, p});
                if (!o_.cost_us) {
                    float feat[16];
                    mlp_features(g.k, g.targets, p, n, post ? 1 : 0, feat);
                    X.insert(X.end(), feat, feat + 16);
                }
            }
        }
        std::vector<double> us(rows.size());
        if (o_.cost_us) {
            for (size_t r = 0; r < rows.size(); ++r) {
                const size_t t = rows[r].first;
                const uint64_t mask = todo[t] & (kPostKey - 1);
                const int path = rows[r].second | ((todo[t] & kPostKey) ? SV_PATH_POST_PHASES : 0);
                us[r] = o_.cost_us(__builtin_popcountll(mask), tg[t].data(), path, (int)(todo[t] >> 56), o_.cost_ctx);
                if (!(us[r] >= 0.0) || !std::isfinite(us[r])) {
                    set_error("sv_fuse_circuit: the cost function returned %g", us[r]);
                    return SV_EINVAL;
                }
            }
        } else {
            SV_TRY(mlp_predict_us(const_cast<sv_mlp *>(o_.model), X.data(), (int)rows.size(), us.data()));
        }
        std::vector<char> seen(todo.size(), 0);
        for (size_t r = 0; r < rows.size(); ++r) {
            auto &k = known_[todo[rows[r].first]];
            if (!seen[rows[r].first] || us[r] < k.first) k = {us[r], rows[r].second};
            seen[rows[r].first] = 1;
        }
        return SV_OK;
    }
    double us(uint64_t key) const { return known_.at(key).first; }
    int path(uint64_t key) const { return known_.at(key).second; }

private:
    const sv_fuse_opts &o_;
    std::unordered_map<uint64_t, std::pair<double, int>> known_;
};

// A candidate partition for the learned search: blocks in order, the light-cone part first.  A
// start from a basis state (sv_init_apply) runs the light-cone part on the small state of the
// qubits that part names (a_mask), with targets renumbered inside it: those blocks are costed on
// that state.
struct Merge;
struct Candidate {
    std::vector<Block> blocks;
    size_t split_at = 0;   // blocks before this index are the light-cone part
    uint64_t a_mask = 0;   // qubits the light-cone part names (0 without a split)
    int n = 0;             // full state's qubits
    // how it was made, to rebuild the winner with matrix expressions: gate order, light-cone split
    // (first / rest parts, or none), max size, closing rule, then the merges of each round
    const std::vector<Dense> *order = nullptr;
    const std::vector<Dense> *first = nullptr, *rest = nullptr;
    int k = 0, rule = 0;
    std::vector<std::vector<Merge>> merges;

    // cost key of block i's gate if it had qubit set `mask`
    uint64_t key(size_t i, uint64_t mask) const
    {
        if (i >= split_at || !a_mask) return cost_key(mask, n);
        uint64_t r = 0;
        int b = 0;
        for (int q = 0; q < 64; ++q)
            if ((a_mask >> q) & 1) {
                if ((mask >> q) & 1) r |= uint64_t(1) << b;
                ++b;
            }
        return cost_key(r, b);
    }
};

// One merge of blocks i < j into a block over the union u, placed at pos (i: block j moves back
// over the blocks between them; j: block i moves forward), predicted to save `gain` microseconds.
struct Merge {
    int i, j, pos;
    uint64_t u;
    double gain;
};

constexpr int kMergeWindow = 32;       // blocks apart at most
constexpr double kMergeMargin = 0.02;  // a merge must save 2% of the two blocks' predicted time
constexpr double kMergeWithin = 0.15;  // candidates within 15% of the best predicted time are merged
constexpr int kMergeRounds = 6;
constexpr int kLightConeTries = 4;     // learned mode also scores light cones of m - 1 .. m - 4 qubits

// Every merge allowed in c: the union has at most max_k qubits, neither block is controlled, both
// lie in the same part, and one of them commutes with every block between them (no shared qubit).
std::vector<Merge> merge_options(const Candidate &c, int max_k)
{
    std::vector<Merge> out;
    const int nb = (int)c.blocks.size();
    std::vector<uint64_t> m(nb);
    for (int i = 0; i < nb; ++i) m[i] = block_mask(c.blocks[i]);
    for (int i = 0; i < nb; ++i) {
        if (c.blocks[i].cmask) continue;
        uint64_t between = 0;   // union of the blocks strictly between i and j
        for (int j = i + 1; j < nb && j <= i + kMergeWindow; ++j) {
            if ((size_t)i < c.split_at && (size_t)j >= c.split_at) break;
            if (!c.blocks[j].cmask) {
                const uint64_t u = m[i] | m[j];
                if (__builtin_popcountll(u) <= max_k) {
                    if (!(between & m[j])) out.push_back(Merge{i, j, i, u, 0.0});
                    else if (!(between & m[i])) out.push_back(Merge{i, j, j, u, 0.0});
                }
            }
            between |= m[j];
        }
    }
    return out;
}

// Applies the chosen merges (pairwise disjoint index ranges) to c.
void apply_merges(Candidate &c, const std::vector<Merge> &ms, int n_qubits)
{
    const int nb = (int)c.blocks.size();
    std::vector<int> at_pos(nb, -1), dropped(nb, 0);
    for (size_t t = 0; t < ms.size(); ++t) {
        at_pos[ms[t].pos] = (int)t;
        dropped[ms[t].pos == ms[t].i ? ms[t].j : ms[t].i] = 1;
    }
    std::vector<Block> out;
    out.reserve(nb);
    size_t split = 0;
    for (int b = 0; b < nb; ++b) {
        if ((size_t)b == c.split_at) split = out.size();
        if (dropped[b]) continue;
        if (at_pos[b] < 0) {
            out.push_back(std::move(c.blocks[b]));
            continue;
        }
        const Merge &mg = ms[(size_t)at_pos[b]];
        Block &a = c.blocks[mg.i];   // earlier in the circuit: its matrix acts first
        Block &z = c.blocks[mg.j];
        Block nbk;
        for (int q = 0; q < n_qubits; ++q)
            if ((mg.u >> q) & 1) nbk.qubits.push_back(q);
        if (a.node) {   // planned candidates carry no matrix expressions
            nbk.node = nbk.qubits == a.qubits ? std::move(a.node) : new_node(nbk.qubits, std::move(a.node));
            nbk.node->ops.push_back(MatOp{{}, {}, std::move(z.node)});
        }
        nbk.n_src = a.n_src + z.n_src;
        nbk.created = a.created;
        out.push_back(std::move(nbk));
    }
    if (c.split_at >= (size_t)nb) split = out.size();
    c.blocks.swap(out);
    c.split_at = c.split_at == 0 ? 0 : split;
}

// Cost-guided merging of every candidate: rounds in which each candidate takes, largest predicted
// saving first, merges whose index ranges do not overlap (a merge then cannot invalidate
// another's commutation check), until no allowed merge is predicted to save time.
int merge_search(std::vector<Candidate> &cands, GateCost &cost, int n_qubits, int max_k)
{
    for (int round = 0; round < kMergeRounds; ++round) {
        std::vector<std::vector<Merge>> opts(cands.size());
        std::vector<uint64_t> need;
        for (size_t c = 0; c < cands.size(); ++c) {
            const Candidate &cd = cands[c];
            opts[c] = merge_options(cd, max_k);
            for (const Merge &m : opts[c]) {
                need.push_back(cd.key((size_t)m.i, m.u));
                need.push_back(cd.key((size_t)m.i, block_mask(cd.blocks[m.i])));
                need.push_back(cd.key((size_t)m.j, block_mask(cd.blocks[m.j])));
            }
        }
        SV_TRY(cost.ensure(need));
        bool any = false;
        for (size_t c = 0; c < cands.size(); ++c) {
            const Candidate &cd = cands[c];
            std::vector<Merge> good;
            for (Merge m : opts[c]) {
                const double two = cost.us(cd.key((size_t)m.i, block_mask(cd.blocks[m.i]))) +
                                   cost.us(cd.key((size_t)m.j, block_mask(cd.blocks[m.j])));
                m.gain = two - cost.us(cd.key((size_t)m.i, m.u));   // both blocks lie in the same part
                if (m.gain > kMergeMargin * two) good.push_back(m);
            }
            std::sort(good.begin(), good.end(), [](const Merge &a, const Merge &b) {
                return a.gain != b.gain ? a.gain > b.gain : (a.i != b.i ? a.i < b.i : a.j < b.j);
            });
            std::vector<char> used(cands[c].blocks.size(), 0);
            std::vector<Merge> pick;
            for (const Merge &m : good) {
                bool free_range = true;
                for (int b = m.i; b <= m.j && free_range; ++b) free_range = !used[(size_t)b];
                if (!free_range) continue;
                for (int b = m.i; b <= m.j; ++b) used[(size_t)b] = 1;
                pick.push_back(m);
            }
            if (!pick.empty()) {
                apply_merges(cands[c], pick, n_qubits);
                cands[c].merges.push_back(std::move(pick));
                any = true;
            }
        }
        if (!any) break;
    }
    return SV_OK;
}

// ------------------------------------------------------------------ post-phase fusion
//
// One fused gate open at a time, its gates kept in order and multiplied out when it closes.  A
// diagonal gate on qubits a (in the open gate, which has no room for b) and b (outside) splits
// into its constant and linear parts (into the open gate for a; a diagonal gate of its own on b,
// held until b's next gate) and its pair part theta x_a x_b: a post-phase term of the open gate
// (it comes after the gate's gates on a and before anything on b).  Rules that keep the order:
// a dense gate on a qubit with a post term (either side) ends the open gate, unless its qubits
// fit and take the term's outside qubit in (then the term becomes an ordinary gate of the open
// gate, appended: it commutes with everything since it was made); held diagonal gates on other
// qubits are emitted before the next gate that touches their qubits.  A closed gate that cannot
// carry post terms on the tensor cores (it must be a 6-qubit gate with at most two targets below
// qubit 5, not both 0 and 1 among them) is first widened with the terms' outside qubits (the
// terms become ordinary gates), then with idle qubits of at least 5; failing that, its terms
// follow it as diagonal fused gates.  A run of at least kMinSwapRun consecutive SWAP gates on
// disjoint qubits becomes one swap network (SV_PATH_SWAPS): the open gate is emitted first if it
// or its terms touch the run's qubits, held gates on them likewise, and the run stays open until a
// gate on one of its qubits arrives (gates on other qubits commute with it).
FusedGate block_to_gate(Block &b);

struct PhaseBlock {
    std::vector<int> qubits;                                      // ascending
    std::vector<std::pair<std::vector<int>, std::vector<cplx>>> ops;   // in order: (qubits, matrix)
    std::vector<FusedGate::PostTerm> post;                        // j = the block qubit (not an index yet)
    int n_src = 0;
    uint64_t mask() const
    {
        uint64_t m = 0;
        for (int q : qubits) m |= uint64_t(1) << q;
        return m;
    }
};

bool is_diag(const std::vector<cplx> &m, size_t d)
{
    for (size_t r = 0; r < d; ++r)
        for (size_t c = 0; c < d; ++c)
            if (r != c && std::abs(m[r * d + c]) > 1e-12) return false;
    return true;
}

// A SWAP gate: two qubits, no controls, the matrix exchanging |01> and |10>.
bool is_swap(const Dense &d)
{
    if (d.cmask || d.q.size() != 2 || d.m.size() != 16) return false;
    for (size_t r = 0; r < 4; ++r)
        for (size_t c = 0; c < 4; ++c) {
            const bool one = (r == 0 && c == 0) || (r == 3 && c == 3) || (r == 1 && c == 2) || (r == 2 && c == 1);
            if (std::abs(d.m[r * 4 + c] - cplx(one ? 1.0 : 0.0)) > 1e-12) return false;
        }
    return true;
}

constexpr int kMinSwapRun = 3;   // consecutive disjoint SWAP gates that become one swap network

bool post_capable(const std::vector<int> &q)
{
    if (q.size() != 6) return false;
    int nlow = 0;
    for (int x : q) nlow += x < 5;
    const bool v4 = q[0] == 0 && q[1] == 1;
    return nlow <= 2 && !v4;
}

std::vector<FusedGate> phase_partition(const std::vector<Dense> &dense, int n_qubits, int max_k, int precision, int tc_min_k)
{
    std::vector<FusedGate> out;
    PhaseBlock cur;
    std::vector<Dense> held;   // diagonal gates off the open block (src 0: a factor split off a gate)
    auto emit_block = [&](PhaseBlock &b) {
        if (b.qubits.empty()) return;
        // widen a block that holds post terms until it can carry them
        if (!b.post.empty() && !post_capable(b.qubits)) {
            std::vector<int> q = b.qubits;
            for (const auto &t : b.post)
                if ((int)q.size() < 6 && std::find(q.begin(), q.end(), t.q) == q.end()) q.push_back(t.q);
            for (int x = n_qubits - 1; x >= 5 && (int)q.size() < 6; --x)
                if (std::find(q.begin(), q.end(), x) == q.end()) q.push_back(x);
            std::sort(q.begin(), q.end());
            if ((int)q.size() <= max_k && post_capable(q)) {
                b.qubits = q;
                std::vector<FusedGate::PostTerm> keep;
                for (const auto &t : b.post) {
                    if (std::find(q.begin(), q.end(), t.q) != q.end()) {
                        // both qubits inside now: an ordinary diagonal gate, after the others
                        const std::vector<cplx> d = {1.0, 1.0, 1.0, std::polar(1.0, t.theta)};
                        b.ops.push_back({{t.j, t.q}, d});
                    } else {
                        keep.push_back(t);
                    }
                }
                b.post = keep;
            }
        }
        PhaseBlock &B = b;
        std::vector<cplx> M = identity(size_t(1) << B.qubits.size());
        for (const auto &op : B.ops) left_multiply(M, B.qubits, op.second, op.first);
        Block blk;
        blk.qubits = B.qubits;
        blk.mat = std::move(M);
        blk.n_src = B.n_src;
        FusedGate fg = block_to_gate(blk);
        fg.path = classify_path(fg, n_qubits, precision, tc_min_k, SV_PATH_AUTO);
        const bool carry = !B.post.empty() && post_capable(B.qubits) && fg.path != SV_PATH_LOW &&
                           fg.path != SV_PATH_HIGH && fg.path != SV_PATH_MIXED;
        std::vector<FusedGate::PostTerm> rest;
        for (const auto &t : B.post) {
            if (carry) {
                const int j = int(std::find(B.qubits.begin(), B.qubits.end(), t.j) - B.qubits.begin());
                fg.post.push_back(FusedGate::PostTerm{j, t.q, t.theta});
            } else {
                rest.push_back(t);
            }
        }
        out.push_back(std::move(fg));
        // terms the gate cannot carry: diagonal fused gates after it, greedily packed
        if (!rest.empty()) {
            std::vector<Dense> dd;
            for (const auto &t : rest) {
                Dense d;
                d.q = {t.j, t.q};
                d.m = {1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, std::polar(1.0, t.theta)};
                d.src = 0;   // its input gate is counted in the gate it followed
                dd.push_back(std::move(d));
            }
            std::vector<Block> bl = greedy_partition(dd, n_qubits, max_k);
            materialize(bl, false);
            for (Block &x : bl) {
                FusedGate g = block_to_gate(x);
                g.path = classify_path(g, n_qubits, precision, tc_min_k, SV_PATH_AUTO);
                out.push_back(std::move(g));
            }
        }
        b = PhaseBlock{};
    };
    auto emit_held = [&](uint64_t touching) {   // held diagonal gates on these qubits, packed
        std::vector<Dense> keep, dd;
        for (Dense &h : held) {
            uint64_t m = 0;
            for (int q : h.q) m |= uint64_t(1) << q;
            (m & touching ? dd : keep).push_back(std::move(h));
        }
        held.swap(keep);
        if (dd.empty()) return;
        std::vector<Block> bl = greedy_partition(dd, n_qubits, max_k);
        materialize(bl, false);
        for (Block &x : bl) {
            FusedGate g = block_to_gate(x);
            g.path = classify_path(g, n_qubits, precision, tc_min_k, SV_PATH_AUTO);
            out.push_back(std::move(g));
        }
    };
    auto post_in = [&]() {
        uint64_t m = 0;
        for (const auto &t : cur.post) m |= uint64_t(1) << t.j;
        return m;
    };
    auto post_out = [&]() {
        uint64_t m = 0;
        for (const auto &t : cur.post) m |= uint64_t(1) << t.q;
        return m;
    };
    // qubits newly in the open block take its post terms on them in as ordinary gates
    auto absorb_terms = [&](uint64_t newq) {
        std::vector<FusedGate::PostTerm> keep;
        for (const auto &t : cur.post) {
            if ((newq >> t.q) & 1) {
                const std::vector<cplx> d = {1.0, 1.0, 1.0, std::polar(1.0, t.theta)};
                cur.ops.push_back({{t.j, t.q}, d});
            } else {
                keep.push_back(t);
            }
        }
        cur.post = keep;
    };
    // swap networks: runs of at least kMinSwapRun consecutive SWAP gates on disjoint qubits (a
    // state of at least 10 qubits) are applied as one in-place pass; a run stays open until a gate
    // on one of its qubits arrives (gates on other qubits commute with it)
    std::vector<int> run_id(dense.size(), -1);
    if (n_qubits >= 10) {
        size_t i = 0;
        int id = 0;
        while (i < dense.size()) {
            size_t j = i;
            uint64_t m = 0;
            while (j < dense.size() && is_swap(dense[j])) {
                const uint64_t q = (uint64_t(1) << dense[j].q[0]) | (uint64_t(1) << dense[j].q[1]);
                if (m & q) break;
                m |= q;
                ++j;
            }
            if (j - i >= (size_t)kMinSwapRun) {
                for (size_t t = i; t < j; ++t) run_id[t] = id;
                ++id;
                i = j;
            } else {
                i = std::max(j, i + 1);
            }
        }
    }
    FusedGate run;
    int run_open = -1;
    auto emit_run = [&]() {
        if (run_open < 0) return;
        run.path = SV_PATH_SWAPS;
        run.k = 0;
        run.mask_lo = (uint32_t)(run.mask & 0xffffffffull);
        out.push_back(std::move(run));
        run = FusedGate{};
        run_open = -1;
    };
    auto add_to_cur = [&](const std::vector<int> &q, const std::vector<cplx> &m, int src) {
        uint64_t newq = 0;
        for (int x : q)
            if (std::find(cur.qubits.begin(), cur.qubits.end(), x) == cur.qubits.end()) {
                cur.qubits.push_back(x);
                newq |= uint64_t(1) << x;
            }
        std::sort(cur.qubits.begin(), cur.qubits.end());
        absorb_terms(newq);
        cur.ops.push_back({q, m});
        cur.n_src += src;
    };
    for (size_t di = 0; di < dense.size(); ++di) {
        const Dense &d = dense[di];
        uint64_t gm = 0;
        for (int x : d.q) gm |= uint64_t(1) << x;
        if (run_open >= 0 && ((run_id[di] >= 0 && run_id[di] != run_open) || ((gm | d.cmask) & run.mask))) emit_run();
        if (run_id[di] >= 0) {   // a SWAP of a run: after everything before it on its qubits
            if ((cur.mask() | post_out()) & gm) emit_block(cur);
            emit_held(gm);
            run_open = run_id[di];
            run.swaps.push_back({std::min(d.q[0], d.q[1]), std::max(d.q[0], d.q[1])});
            run.mask |= gm;
            run.n_src += d.src;
            continue;
        }
        if (d.cmask) {   // a controlled gate kept whole: on its own, after what touches its qubits
            const uint64_t all = gm | d.cmask;
            if ((cur.mask() | post_out()) & all) emit_block(cur);
            emit_held(all);
            Block cb = controlled_block(d, true);
            cb.mat = evaluate(*cb.node);
            FusedGate g = block_to_gate(cb);
            g.path = SV_PATH_CONTROLLED;
            out.push_back(std::move(g));
            continue;
        }
        const size_t dim = d.m.size() == 0 ? 0 : (size_t)std::llround(std::sqrt((double)d.m.size()));
        const bool diag = is_diag(d.m, dim);
        const uint64_t cm = cur.mask();
        const int unionk = __builtin_popcountll(cm | gm);
        if (diag && d.q.size() == 2 && (cm & gm) && unionk > max_k && !(post_out() & (cm & gm))) {
            // one qubit in the open block, one outside: constant and linear parts, and a post term
            const int a = (cm >> d.q[0]) & 1 ? d.q[0] : d.q[1];
            const int b = a == d.q[0] ? d.q[1] : d.q[0];
            const int ba = a == d.q[0] ? 0 : 1;   // local bit of a in d's index
            const cplx d00 = d.m[0], da = d.m[(size_t)(5 * (1 << ba))], db = d.m[(size_t)(5 * (1 << (1 - ba)))], d11 = d.m[15];
            // d = d00 * diag_a(1, da/d00) * diag_b(1, db/d00) * exp(i theta x_a x_b)
            const double theta = std::arg(d11 * d00 / (da * db));
            add_to_cur({a}, {d00, 0.0, 0.0, da}, 1);   // constant and the linear part on a
            if (std::abs(db / d00 - 1.0) > 1e-15) {
                Dense hb;
                hb.q = {b};
                hb.m = {1.0, 0.0, 0.0, db / d00};
                hb.src = 0;
                held.push_back(std::move(hb));
            }
            cur.post.push_back(FusedGate::PostTerm{a, b, theta});
            continue;
        }
        if (diag && !(cm & gm) && unionk > max_k) {   // a diagonal gate off the open block: held
            held.push_back(d);
            continue;
        }
        // dense gates (and diagonal ones that fit): held diagonal gates on their qubits go first
        const bool conflict = (gm & post_in()) != 0;
        const bool fits = unionk <= max_k;
        if (conflict || !fits) emit_block(cur);
        // held gates touching g: into the open block when they fit with g, else before it
        uint64_t hm = 0;
        for (const Dense &h : held)
            for (int x : h.q)
                if ((gm >> x) & 1) {
                    for (int y : h.q) hm |= uint64_t(1) << y;
                }
        if (hm) {
            if (__builtin_popcountll(cur.mask() | gm | hm) <= max_k && !(hm & post_in())) {
                std::vector<Dense> keep;
                for (Dense &h : held) {
                    uint64_t m = 0;
                    for (int y : h.q) m |= uint64_t(1) << y;
                    if (m & gm) add_to_cur(h.q, h.m, h.src);
                    else keep.push_back(std::move(h));
                }
                held.swap(keep);
            } else {
                emit_block(cur);
                emit_held(gm);
            }
        }
        add_to_cur(d.q, d.m, 1);
    }
    emit_block(cur);
    emit_held(~uint64_t(0));
    emit_run();
    return out;
}

bool is_unitary(const std::vector<cplx> &U, size_t d, double tol)
{
    for (size_t i = 0; i < d; ++i)
        for (size_t j = 0; j < d; ++j) {
            cplx acc = 0.0;
            for (size_t r = 0; r < d; ++r) acc += std::conj(U[r * d + i]) * U[r * d + j];
            if (std::abs(acc - (i == j ? cplx(1.0) : cplx(0.0))) > tol) return false;
        }
    return true;
}

// Round a finished block into a fused gate (fp64 matrix kept, fp32 copies rounded once).
FusedGate block_to_gate(Block &b)
{
    FusedGate fg;
    fg.k = (int)b.qubits.size();
    for (int j = 0; j < fg.k; ++j) {
        fg.targets[j] = b.qubits[j];
        fg.mask |= uint64_t(1) << b.qubits[j];
        if (b.qubits[j] < 32) fg.mask_lo |= 1u << b.qubits[j];
    }
    fg.n_src = b.n_src;
    fg.cmask = b.cmask;
    fg.mat = std::move(b.mat);
    const size_t d2 = fg.mat.size();
    fg.ur.resize(d2);
    fg.ui.resize(d2);
    for (size_t i = 0; i < d2; ++i) {
        fg.ur[i] = (float)fg.mat[i].real();
        fg.ui[i] = (float)fg.mat[i].imag();
    }
    return fg;
}

}  // namespace

std::vector<FusedGate> refuse_gates(const std::vector<const FusedGate *> &in, int n_qubits, int max_k)
{
    std::vector<Dense> dense(in.size());
    for (size_t i = 0; i < in.size(); ++i) {
        dense[i].q.assign(in[i]->targets, in[i]->targets + in[i]->k);
        dense[i].m = in[i]->mat;
    }
    std::vector<Block> blocks = greedy_partition(dense, n_qubits, max_k);
    materialize(blocks, false);
    std::vector<FusedGate> out;
    out.reserve(blocks.size());
    for (Block &b : blocks) {
        out.push_back(block_to_gate(b));
        out.back().path = SV_PATH_AUTO;
    }
    return out;
}

int classify_path(const FusedGate &g, int n, int precision, int tc_min_k, int force_path)
{
    if (g.cmask) return SV_PATH_CONTROLLED;
    if (force_path != SV_PATH_AUTO) return force_path;
    // tensor cores for 4..6-qubit gates of states with at least 2^k blocks of 32 amplitudes
    if (precision != SV_PREC_FP32 && g.k >= tc_min_k && g.k >= 4 && n >= g.k + 5)
        return precision == SV_PREC_TF32 ? SV_PATH_TC_TF32 : SV_PATH_TC_BF16X3;
    bool any_low = false, any_high = false;
    for (int j = 0; j < g.k; ++j) (g.targets[j] < 5 ? any_low : any_high) = true;
    if (!any_high) return SV_PATH_LOW;
    if (!any_low) return SV_PATH_HIGH;
    return SV_PATH_MIXED;
}

}  // namespace svg

using namespace svg;

extern "C" int sv_fuse_circuit(const sv_gate *gates, int n_gates, int n_qubits,
                               const sv_fuse_opts *opts_in, sv_fused **out)
{
    clear_error();
    if (!out) { set_error("sv_fuse_circuit: out is NULL"); return SV_EINVAL; }
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS) {
        set_error("sv_fuse_circuit: n_qubits=%d outside [1, %d]", n_qubits, SV_MAX_QUBITS);
        return SV_EINVAL;
    }
    if (n_gates < 0 || (n_gates > 0 && !gates)) { set_error("sv_fuse_circuit: bad gate array"); return SV_EINVAL; }
    sv_fuse_opts opts{};
    opts.max_k = 4;
    if (opts_in) opts = *opts_in;
    if (opts.max_k == 0) opts.max_k = 4;
    if (opts.tc_min_k == 0) opts.tc_min_k = 5;
    if (opts.max_k < 1 || opts.max_k > SV_MAX_K) { set_error("sv_fuse_circuit: max_k=%d outside [1, 6]", opts.max_k); return SV_EINVAL; }
    if (opts.precision < SV_PREC_FP32 || opts.precision > SV_PREC_BF16X3) { set_error("sv_fuse_circuit: bad precision %d", opts.precision); return SV_EINVAL; }
    if (opts.tc_min_k < 1 || opts.tc_min_k > SV_MAX_K) { set_error("sv_fuse_circuit: tc_min_k=%d outside [1, 6]", opts.tc_min_k); return SV_EINVAL; }
    if (opts.force_path < SV_PATH_AUTO || opts.force_path > SV_PATH_TC_BF16X3) { set_error("sv_fuse_circuit: bad force_path"); return SV_EINVAL; }
    if (opts.mode != SV_FUSE_GREEDY && opts.mode != SV_FUSE_LEARNED && opts.mode != SV_FUSE_NONE && opts.mode != SV_FUSE_PHASES) {
        set_error("sv_fuse_circuit: bad mode");
        return SV_EINVAL;
    }
    if (opts.mode == SV_FUSE_PHASES && (opts.precision == SV_PREC_FP32 || opts.start_qubits != 0 || opts.force_path != SV_PATH_AUTO)) {
        set_error("sv_fuse_circuit: SV_FUSE_PHASES needs tensor-core precision, no start_qubits and no forced path");
        return SV_EINVAL;
    }
    if (opts.start_qubits < 0 || opts.start_qubits > kMaxStartQubits) { set_error("sv_fuse_circuit: start_qubits=%d outside [0, %d]", opts.start_qubits, kMaxStartQubits); return SV_EINVAL; }

    // ---- validate and densify every input gate (controls folded into the matrix where they fit
    // the fusion size; otherwise small gates stay controlled)
    std::vector<Dense> dense;
    try { dense.resize(size_t(n_gates)); } catch (const std::bad_alloc &) { set_error("sv_fuse_circuit: out of host memory"); return SV_ENOMEM; }
    const int fold_limit = opts.mode == SV_FUSE_NONE ? SV_MAX_K : opts.max_k;
    for (int gi = 0; gi < n_gates; ++gi) {
        const sv_gate &g = gates[gi];
        if (g.k < 1 || g.k > SV_MAX_K || g.n_controls < 0 || g.n_controls > SV_MAX_CONTROLS || !g.mat) {
            set_error("sv_fuse_circuit: gate %d has k=%d, n_controls=%d (need 1 <= k <= 6, 0 <= controls <= %d) or no matrix", gi, g.k,
                      g.n_controls, SV_MAX_CONTROLS);
            return SV_EINVAL;
        }
        const bool keep_controlled = g.n_controls > 0 && g.k + g.n_controls > fold_limit && g.k <= kMaxControlledK;
        if (!keep_controlled && g.k + g.n_controls > SV_MAX_K) {
            set_error("sv_fuse_circuit: gate %d has k=%d and %d controls: a controlled gate keeps at most %d targets, "
                      "a folded one at most 6 qubits", gi, g.k, g.n_controls, kMaxControlledK);
            return SV_EINVAL;
        }
        uint64_t used = 0;
        std::vector<int> q;
        for (int j = 0; j < g.k + g.n_controls; ++j) {
            int qq = j < g.k ? g.targets[j] : g.controls[j - g.k];
            if (qq < 0 || qq >= n_qubits || ((used >> qq) & 1)) {
                set_error("sv_fuse_circuit: gate %d names qubit %d (out of range or repeated)", gi, qq);
                return SV_EINVAL;
            }
            used |= uint64_t(1) << qq;
            q.push_back(qq);
        }
        const size_t d = size_t(1) << g.k;
        std::vector<cplx> U(d * d);
        for (size_t i = 0; i < d * d; ++i) U[i] = cplx(g.mat[2 * i], g.mat[2 * i + 1]);
        if (!is_unitary(U, d, 1e-8)) {
            set_error("sv_fuse_circuit: gate %d is not unitary (|U^H U - I| > 1e-8)", gi);
            return SV_EUNITARY;
        }
        if (keep_controlled) {
            q.resize(size_t(g.k));
            for (int j = 0; j < g.n_controls; ++j) dense[gi].cmask |= uint64_t(1) << g.controls[j];
            dense[gi].q = q;
            dense[gi].m = std::move(U);
            continue;
        }
        // controlled matrix on local bits (targets..., controls...): U where all controls are 1
        const int kk = g.k + g.n_controls;
        const size_t D = size_t(1) << kk;
        std::vector<cplx> M = identity(D);
        if (g.n_controls > 0) {
            const size_t c_on = ((size_t(1) << g.n_controls) - 1) << g.k;
            for (size_t r = 0; r < d; ++r)
                for (size_t c = 0; c < d; ++c) M[(c_on | r) * D + (c_on | c)] = U[r * d + c];
        } else {
            M = U;
        }
        dense[gi].q = q;
        dense[gi].m = std::move(M);
    }

    // light-cone split for a start from a basis state (at most 28 qubits and fewer than n: the
    // small state sv_init_apply runs them on)
    const int start_m = std::min(opts.start_qubits, std::min(kMaxStartQubits, n_qubits - 1));
    const bool split = opts.start_qubits > 0 && start_m > 0 && opts.mode != SV_FUSE_NONE;
    std::vector<Dense> first, rest;
    if (split) {
        try {
            split_light_cone(dense, start_m, first, rest);
        } catch (const std::bad_alloc &) {
            set_error("sv_fuse_circuit: out of host memory");
            return SV_ENOMEM;
        }
    }

    sv_fused *f = new (std::nothrow) sv_fused();
    if (!f) { set_error("sv_fuse_circuit: out of host memory"); return SV_ENOMEM; }
    f->n = n_qubits;
    f->precision = opts.precision;

    auto finish = [&](Block &b, int path) {
        FusedGate fg = block_to_gate(b);
        fg.path = path >= 0 ? path : classify_path(fg, n_qubits, opts.precision, opts.tc_min_k, opts.force_path);
        f->gates.push_back(std::move(fg));
    };

    try {
        if (opts.mode == SV_FUSE_PHASES) {
            f->gates = phase_partition(dense, n_qubits, opts.max_k, opts.precision, opts.tc_min_k);
        } else if (opts.mode == SV_FUSE_NONE) {
            // one block per input gate, matrix re-expressed over its ascending qubit list
            for (int gi = 0; gi < n_gates; ++gi) {
                if (dense[gi].cmask) {
                    Block cb = controlled_block(dense[gi]);
                    cb.mat = evaluate(*cb.node);
                    finish(cb, -1);
                    continue;
                }
                Block b;
                b.qubits = dense[gi].q;
                std::sort(b.qubits.begin(), b.qubits.end());
                b.mat = identity(size_t(1) << b.qubits.size());
                left_multiply(b.mat, b.qubits, dense[gi].m, dense[gi].q);
                b.n_src = 1;
                finish(b, -1);
            }
        } else if (opts.mode == SV_FUSE_GREEDY || (!opts.cost_us && !mlp_usable(opts.model, kMaxTrustedError))) {
            const int k = opts.mode == SV_FUSE_GREEDY ? opts.max_k : (opts.model ? mlp_fallback_k(opts.model) : opts.max_k);
            size_t split_at = 0;
            std::vector<Block> blocks = partition(dense, split ? &first : nullptr, &rest, n_qubits, k, kCloseOutside, &split_at);
            uint64_t a_mask = 0;
            for (size_t i = 0; i < split_at; ++i) a_mask |= block_mask(blocks[i]);
            f->lazy_limit = __builtin_popcountll(a_mask);
            materialize(blocks, true);
            for (Block &b : blocks) finish(b, -1);
        } else {
            // learned: candidate partitions -- greedy at every max size 2..max_k under each rule
            // for which blocks a gate closes -- each improved by cost-guided merging, then scored
            // by the predicted time of its fused gates (each on its cheapest path); the cheapest
            // candidate wins
            // With a light-cone split (a start from a basis state) the split size is a candidate
            // too: the light cone on m' <= m qubits, its gates costed on the 2^|A| small state.
            // A larger light cone moves more gates off the full state but makes every small-state
            // gate dearer, so smaller ones are scored at the largest fusion size.
            struct Split {
                int m;
                std::vector<Dense> first, rest;
            };
            std::vector<Split> splits;
            if (split) {
                splits.push_back(Split{start_m, first, rest});
                for (int mm = start_m - 1; mm >= std::max(1, start_m - kLightConeTries); --mm) {
                    Split sp{mm, {}, {}};
                    split_light_cone(dense, mm, sp.first, sp.rest);
                    splits.push_back(std::move(sp));
                }
            }
            std::vector<Dense> deferred;
            Split dsplit{start_m, {}, {}};
            if (!defer_diagonals(dense, deferred)) deferred.clear();
            else if (split) split_light_cone(deferred, start_m, dsplit.first, dsplit.rest);
            std::vector<Candidate> cand;
            {   // candidates are planned on qubit sets only (no matrix expressions), on host threads
                auto plan = [&](const std::vector<Dense> *order, const std::vector<Dense> *fp, const std::vector<Dense> *rp, int k, int rule) {
                    Candidate c;
                    c.n = n_qubits;
                    c.order = order;
                    c.first = fp;
                    c.rest = rp;
                    c.k = k;
                    c.rule = rule;
                    cand.push_back(std::move(c));
                };
                const int kmax = std::max(2, opts.max_k);
                for (int k = 2; k <= kmax; ++k)
                    for (int rule = 0; rule < kCloseRules; ++rule)
                        plan(&dense, split ? &splits[0].first : nullptr, split ? &splits[0].rest : nullptr, k, rule);
                for (size_t i = 1; i < splits.size(); ++i) plan(&dense, &splits[i].first, &splits[i].rest, kmax, kCloseOutside);
                if (!deferred.empty())   // the equivalent order with diagonal gates deferred, at every max size
                    for (int k = 2; k <= kmax; ++k)
                        plan(&deferred, split ? &dsplit.first : nullptr, split ? &dsplit.rest : nullptr, k, kCloseOutside);
                host_parallel_for(cand.size(), std::min<size_t>(cand.size(), 8), [&](size_t i) {
                    Candidate &c = cand[i];
                    c.blocks = partition(*c.order, c.first, c.rest, n_qubits, c.k, c.rule, &c.split_at, false);
                    for (size_t j = 0; j < c.split_at; ++j) c.a_mask |= block_mask(c.blocks[j]);
                });
            }
            // identical partitions (different rules often agree) are scored once
            {
                std::vector<Candidate> uniq;
                std::vector<std::vector<uint64_t>> seen;
                for (Candidate &c : cand) {
                    std::vector<uint64_t> key = {c.a_mask, (uint64_t)c.split_at};
                    for (const Block &b : c.blocks) key.push_back(block_mask(b));
                    if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
                    seen.push_back(std::move(key));
                    uniq.push_back(std::move(c));
                }
                cand.swap(uniq);
            }
            GateCost cost(opts);
            auto total = [&](const Candidate &c) {
                double tot = 0.0;
                for (size_t i = 0; i < c.blocks.size(); ++i)   // kept controlled gates: the same in every candidate
                    if (!c.blocks[i].cmask) tot += cost.us(c.key(i, block_mask(c.blocks[i])));
                return tot;
            };
            auto score_all = [&]() -> int {
                std::vector<uint64_t> all;
                for (const Candidate &c : cand)
                    for (size_t i = 0; i < c.blocks.size(); ++i)
                        if (!c.blocks[i].cmask) {
                            all.push_back(c.key(i, block_mask(c.blocks[i])));
                            if (i < c.split_at) all.push_back(cost_key(block_mask(c.blocks[i]), n_qubits));   // its full-state path
                        }
                return cost.ensure(all);
            };
            int rc = score_all();
            if (rc == SV_OK) {
                // merging searches the candidates within kMergeWithin of the best one as it stands
                // (a merge saves at most one gate's time, so far worse partitions cannot catch up)
                double best0 = 0.0;
                for (size_t c = 0; c < cand.size(); ++c) best0 = c == 0 ? total(cand[c]) : std::min(best0, total(cand[c]));
                std::vector<Candidate> near, far;
                for (Candidate &c : cand) (total(c) <= (1.0 + kMergeWithin) * best0 ? near : far).push_back(std::move(c));
                rc = merge_search(near, cost, n_qubits, std::max(2, opts.max_k));
                cand.clear();
                for (Candidate &c : near) cand.push_back(std::move(c));
                for (Candidate &c : far) cand.push_back(std::move(c));
            }
            if (rc == SV_OK) rc = score_all();
            if (rc != SV_OK) { delete f; return rc; }
            size_t best = 0;
            double best_t = 0.0;
            for (size_t c = 0; c < cand.size(); ++c) {
                const double tot = total(cand[c]);
                if (c == 0 || tot < best_t) { best = c; best_t = tot; }
            }
            // the post-phase partition (SV_FUSE_PHASES) as one more candidate, where it can differ
            // from the others: tensor-core precision, six-qubit gates, no light-cone split, and a
            // diagonal two-qubit gate somewhere.  It is made with its matrices (the post terms
            // come from the gates' entries); a gate that carries post-phases is scored as one.
            bool phases = opts.precision != SV_PREC_FP32 && opts.max_k == 6 && !split && opts.force_path == SV_PATH_AUTO;
            if (phases) {
                bool any = false;
                for (const Dense &d : dense)
                    if (d.q.size() == 2 && is_diagonal(d)) any = true;
                phases = any;
            }
            if (phases) {
                std::vector<FusedGate> ph = phase_partition(dense, n_qubits, opts.max_k, opts.precision, opts.tc_min_k);
                // a swap network is one read and one write of the state: scored as a one-qubit
                // gate on the top qubit (the cheapest full pass there is)
                auto key_of = [&](const FusedGate &g) {
                    if (g.path == SV_PATH_SWAPS) return cost_key(uint64_t(1) << (n_qubits - 1), n_qubits);
                    uint64_t m = 0;
                    for (int j = 0; j < g.k; ++j) m |= uint64_t(1) << g.targets[j];
                    return cost_key(m, n_qubits) | (g.post.empty() ? 0 : kPostKey);
                };
                std::vector<uint64_t> keys;
                for (const FusedGate &g : ph)
                    if (!g.cmask) keys.push_back(key_of(g));
                if ((rc = cost.ensure(keys)) != SV_OK) { delete f; return rc; }
                double tot = 0.0;
                for (uint64_t key : keys) tot += cost.us(key);
                if (tot < best_t) {
                    for (FusedGate &g : ph)   // gates without post-phases on their cheapest path
                        if (!g.cmask && g.post.empty() && g.path != SV_PATH_SWAPS) g.path = cost.path(key_of(g));
                    f->gates = std::move(ph);
                    f->lazy_limit = 0;
                    *out = f;
                    return SV_OK;
                }
            }
            f->lazy_limit = __builtin_popcountll(cand[best].a_mask);
            // the winner again, with matrix expressions, and its merges replayed: the same blocks
            const Candidate &w = cand[best];
            Candidate win;
            win.n = n_qubits;
            win.blocks = partition(*w.order, w.first, w.rest, n_qubits, w.k, w.rule, &win.split_at, true);
            win.a_mask = w.a_mask;
            for (const std::vector<Merge> &pick : w.merges) apply_merges(win, pick, n_qubits);
            bool same = win.blocks.size() == w.blocks.size();
            for (size_t i = 0; same && i < w.blocks.size(); ++i) same = block_mask(win.blocks[i]) == block_mask(w.blocks[i]);
            if (!same) { delete f; set_error("sv_fuse_circuit: internal error (learned partition rebuilt differently)"); return SV_EINVAL; }
            materialize(win.blocks, true);
            // each gate's path for the full state (sv_init_apply re-picks it on the small state)
            for (Block &b : win.blocks) finish(b, b.cmask ? SV_PATH_CONTROLLED : cost.path(cost_key(block_mask(b), n_qubits)));
        }
    } catch (const std::bad_alloc &) {
        delete f;
        set_error("sv_fuse_circuit: out of host memory");
        return SV_ENOMEM;
    } catch (const std::exception &e) {   // e.g. no host thread for a candidate partition
        delete f;
        set_error("sv_fuse_circuit: %s", e.what());
        return SV_ENOMEM;
    }
    *out = f;
    return SV_OK;
}

extern "C" int sv_fused_get_post_phases(const sv_fused *f, int i, int max_terms, int *target, int *qubit, double *angle)
{
    clear_error();
    if (!f || i < 0 || i >= (int)f->gates.size() || max_terms < 0) { set_error("sv_fused_get_post_phases: bad argument"); return SV_EINVAL; }
    const std::vector<FusedGate::PostTerm> &post = f->gates[(size_t)i].post;
    for (int t = 0; t < (int)post.size() && t < max_terms; ++t) {
        if (target) target[t] = post[(size_t)t].j;
        if (qubit) qubit[t] = post[(size_t)t].q;
        if (angle) angle[t] = post[(size_t)t].theta;
    }
    return (int)post.size();
}

extern "C" int sv_fused_get_swaps(const sv_fused *f, int i, int max_pairs, int *qubit_a, int *qubit_b)
{
    clear_error();
    if (!f || i < 0 || i >= (int)f->gates.size() || max_pairs < 0) { set_error("sv_fused_get_swaps: bad argument"); return SV_EINVAL; }
    const std::vector<std::pair<int, int>> &sw = f->gates[(size_t)i].swaps;
    for (int t = 0; t < (int)sw.size() && t < max_pairs; ++t) {
        if (qubit_a) qubit_a[t] = sw[(size_t)t].first;
        if (qubit_b) qubit_b[t] = sw[(size_t)t].second;
    }
    return (int)sw.size();
}

extern "C" int sv_fused_count(const sv_fused *f)
{
    return f ? (int)f->gates.size() : SV_EINVAL;
}

extern "C" int sv_fused_get_info(const sv_fused *f, int i, sv_fused_info *info)
{
    clear_error();
    if (!f || !info || i < 0 || i >= (int)f->gates.size()) { set_error("sv_fused_get_info: bad argument"); return SV_EINVAL; }
    const FusedGate &g = f->gates[size_t(i)];
    std::memset(info, 0, sizeof(*info));
    info->k = g.k;
    for (int j = 0; j < g.k; ++j) info->targets[j] = g.targets[j];
    info->path = g.path;
    info->n_source_gates = g.n_src;
    info->control_mask = g.cmask;
    return SV_OK;
}

extern "C" int sv_fused_get_matrix(const sv_fused *f, int i, double *out)
{
    clear_error();
    if (!f || !out || i < 0 || i >= (int)f->gates.size()) { set_error("sv_fused_get_matrix: bad argument"); return SV_EINVAL; }
    const FusedGate &g = f->gates[size_t(i)];
    if (g.path == SV_PATH_SWAPS) { set_error("sv_fused_get_matrix: gate %d is a swap network (sv_fused_get_swaps)", i); return SV_EINVAL; }
    for (size_t e = 0; e < g.mat.size(); ++e) {
        out[2 * e] = g.mat[e].real();
        out[2 * e + 1] = g.mat[e].imag();
    }
    return SV_OK;
}
