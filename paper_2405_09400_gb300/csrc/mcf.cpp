// Host min-cost flow for the flow update, Eq. (MinCostFlow).
//
// The problem is a transportation problem on the neighbourhood graph
// (Def. 3.1): every basic cell i is a source with supply m_i and a sink with
// demand m_i; arc (i -> j) for j in N(i) carries w_ij >= 0 at cost c_bar_ij;
// the divergence constraints of Eq. (div-constraint-single-cell) are the
// supplies and demands. The paper solves it with OR-tools; this is a
// project-written primal network simplex in exact int64 arithmetic:
//
//  * masses are scaled to integers (sum 2^60) and costs to integers (2^40 at the
//    largest |c_bar|); w_ij = m_i * q_ij / M_i maps the integer flow back, so
//    sum_j w_ij = m_i holds to float64 rounding;
//  * the start basis is the stationary flow (w_ii = m_i, Lemma 3.6) completed to
//    a spanning tree by zero-flow arcs s_p -> t_i along a spanning tree of the
//    cell grid; it is strongly feasible, and the leaving arc is chosen by
//    Cunningham's rule (last blocking arc from the apex), which rules out cycling;
//  * entering arcs from a candidate list of arcs with negative reduced cost,
//    refilled by block scans;
//  * the tree is kept in preorder-thread form (parent, thread, reverse thread,
//    subtree size, last node of the subtree): the join of a pivot cycle is found
//    by climbing from the side with the smaller subtree, the cut subtree is
//    re-rooted by relinking O(stem) thread segments, and the potentials of the
//    smaller of the cut subtree and the rest are shifted, walking the thread.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/ddflow.h"

namespace {

int mcf_block = 0;  // entering-arc block size; 0 = sqrt(#arcs)

// The spanning tree is kept in preorder-thread form: thread[x] is the node after
// x in a preorder walk of the tree (cyclic), rev_thread its inverse, succ[x] the
// size of x's subtree and last[x] the last node of x's subtree in that order, so
// every subtree is one contiguous run of the thread.
struct NetworkSimplex {
    int nn = 0;  // nodes: source of cell i = 2i, sink of cell i = 2i + 1 (adjacent in memory)
    int na = 0;  // arcs
    int root = 0;
    std::vector<int> tail, head;
    std::vector<int64_t> cost, flow;
    std::vector<int> parent, parc, thread, rev_thread, succ, last;
    std::vector<int64_t> pot;
    std::vector<int> pu, pv, stem, seg;
    int64_t pivots = 0;
#ifdef MCF_STATS
    int64_t st_refresh = 0, st_path = 0, st_scan = 0, st_degenerate = 0;
#endif

    int64_t rc(int a) const { return cost[a] + pot[tail[a]] - pot[head[a]]; }

    // thread, sizes and last nodes from parent pointers (child lists built here)
    void build_thread() {
        std::vector<int> first_child(nn, -1), next_sib(nn, -1);
        for (int x = nn - 1; x >= 0; --x)
            if (parent[x] >= 0) {
                next_sib[x] = first_child[parent[x]];
                first_child[parent[x]] = x;
            }
        thread.assign(nn, -1);
        rev_thread.assign(nn, -1);
        succ.assign(nn, 1);
        last.assign(nn, -1);
        std::vector<int> order, st;
        order.reserve(nn);
        st.push_back(root);
        while (!st.empty()) {
            int x = st.back();
            st.pop_back();
            order.push_back(x);
            std::vector<int> ch;
            for (int c = first_child[x]; c >= 0; c = next_sib[c]) ch.push_back(c);
            for (int k = (int)ch.size() - 1; k >= 0; --k) st.push_back(ch[k]);
        }
        for (int k = 0; k < nn; ++k) {
            thread[order[k]] = order[(k + 1) % nn];
            rev_thread[order[(k + 1) % nn]] = order[k];
        }
        for (int k = nn - 1; k >= 0; --k) {
            int x = order[k];
            if (parent[x] >= 0) succ[parent[x]] += succ[x];
        }
        for (int k = 0; k < nn; ++k) {
            int x = order[k];
            last[x] = order[k + succ[x] - 1];
        }
    }

    // potentials of the whole tree from the root, tree arcs priced at 0
    void price_tree() {
        pot[root] = 0;
        for (int x = thread[root]; x != root; x = thread[x]) {
            const int p = parent[x], a = parc[x];
            pot[x] = (tail[a] == p) ? pot[p] + cost[a] : pot[p] - cost[a];
        }
    }

    bool pivot(int a) {
        const int u = tail[a], v = head[a];
        // join of the two tree paths: climb from the side with the smaller subtree
        // (an ancestor's subtree is strictly larger); pu / pv hold the nodes
        // strictly below the join on each side, from u resp. v upwards
        pu.clear();
        pv.clear();
        int x = u, y = v;
        while (x != y) {
            if (succ[x] < succ[y]) {
                pu.push_back(x);
                x = parent[x];
            } else {
                pv.push_back(y);
                y = parent[y];
            }
        }
        const int join = x;
        // cycle join -> u, a, v -> join: on the u path arcs pointing up are
        // backward (blocking), on the v path arcs pointing down. theta is the
        // least flow on a blocking arc, and the leaving arc the last blocking arc
        // with that flow in cycle order from the join (keeps the basis strongly
        // feasible, no cycling): one walk in reverse cycle order (the v path from
        // the join down, then the u path from u up) keeping the first minimum
        int64_t theta = INT64_MAX;
        int q = -1;
        bool on_v = false;
        for (int k = (int)pv.size() - 1; k >= 0; --k) {
            const int z = pv[k], e = parc[z];
            if (head[e] == z && flow[e] < theta) {
                theta = flow[e];
                q = z;
                on_v = true;
            }
        }
        for (int k = 0; k < (int)pu.size(); ++k) {
            const int z = pu[k], e = parc[z];
            if (tail[e] == z && flow[e] < theta) {
                theta = flow[e];
                q = z;
                on_v = false;
            }
        }
        if (theta == INT64_MAX) return false;  // unbounded (cannot happen here)
#ifdef MCF_STATS
        st_path += pu.size() + pv.size();
        if (theta == 0) ++st_degenerate;
#endif
        if (q < 0) return false;
        if (theta > 0) {
            for (int z : pu) {
                int e = parc[z];
                flow[e] += (tail[e] == z) ? -theta : theta;
            }
            for (int z : pv) {
                int e = parc[z];
                flow[e] += (head[e] == z) ? -theta : theta;
            }
            flow[a] += theta;
        }
        // the subtree S of q is cut at its parent and hung at the endpoint u_in
        // of a inside S below the other endpoint v_in; its potentials shift by
        // delta (only differences matter: the smaller of S and the rest moves)
        const int u_in = on_v ? v : u, v_in = on_v ? u : v;
        const int64_t delta = on_v ? rc(a) : -rc(a);
        const int p_out = parent[q];
        const int nS = succ[q];
        // stem u_in = w0, w1, ..., wk = q (old ancestors of u_in inside S)
        stem.clear();
        for (int z = u_in; z != q; z = parent[z]) stem.push_back(z);
        stem.push_back(q);
        const int k = (int)stem.size() - 1;
        // 1. take S out of the thread (old links), fix sizes / last nodes above it
        const int lastS = last[q], before = rev_thread[q], after = thread[lastS];
        thread[before] = after;
        rev_thread[after] = before;
        for (int z = p_out; z != join; z = parent[z]) succ[z] -= nS;
        for (int z = p_out; z >= 0 && last[z] == lastS; z = parent[z]) last[z] = before;
        // 2. the new preorder of S rooted at w0: the old block of w0, then for
        //    i = 1..k the rest of w_i's old block (the part before w_{i-1}'s
        //    block, then the part after it). All old links are read first.
        seg.resize(3 * (size_t)(k + 1));
        for (int i = 1; i <= k; ++i) {
            const int wi = stem[i], wp = stem[i - 1];
            seg[3 * i] = rev_thread[wp];                                  // end of the part before
            seg[3 * i + 1] = last[wp] != last[wi] ? thread[last[wp]] : -1;  // start of the part after
            seg[3 * i + 2] = last[wi];                                    // its end
        }
        int tailS = last[stem[0]];
        for (int i = 1; i <= k; ++i) {
            const int wi = stem[i];
            thread[tailS] = wi;
            rev_thread[wi] = tailS;
            tailS = seg[3 * i];
            if (seg[3 * i + 1] >= 0) {
                thread[tailS] = seg[3 * i + 1];
                rev_thread[seg[3 * i + 1]] = tailS;
                tailS = seg[3 * i + 2];
            }
        }
        // sizes and last nodes of the stem, parents / tree arcs reversed along it
        const int nk = succ[q];
        for (int i = k; i >= 1; --i) succ[stem[i]] = nk - succ[stem[i - 1]];
        succ[stem[0]] = nk;
        for (int i = 0; i <= k; ++i) last[stem[i]] = tailS;
        for (int i = k; i >= 1; --i) {
            parent[stem[i]] = stem[i - 1];
            parc[stem[i]] = parc[stem[i - 1]];
        }
        parent[u_in] = v_in;
        parc[u_in] = a;
        // 3. S after v_in in the thread; sizes / last nodes above v_in
        const int nxt = thread[v_in];
        const bool v_leaf = last[v_in] == v_in;
        thread[v_in] = u_in;
        rev_thread[u_in] = v_in;
        thread[tailS] = nxt;
        rev_thread[nxt] = tailS;
        for (int z = v_in; z != join; z = parent[z]) succ[z] += nS;
        if (v_leaf)
            for (int z = v_in; z >= 0 && last[z] == v_in; z = parent[z]) last[z] = tailS;
        // 4. potentials
        if (2 * nS <= nn) {
            int z = u_in;
            for (int t = 0; t < nS; ++t, z = thread[z]) pot[z] += delta;
        } else {
            int z = thread[tailS];
            for (int t = 0; t < nn - nS; ++t, z = thread[z]) pot[z] -= delta;
        }
#ifdef MCF_STATS
        st_refresh += std::min(nS, nn - nS);
#endif
        ++pivots;
        return true;
    }

    // Entering arcs by a candidate list: a major pass scans blocks of arcs (in a
    // rotating order) until it has collected up to kCand arcs of negative reduced
    // cost; minor passes re-price only the list and pivot on its most negative
    // arc, dropping arcs that are no longer eligible, until the list is empty.
    // Tree arcs price at exactly 0 (integer potentials) and are never taken.
    // The list length grows with the arc count (na/128, between 256 and 4096):
    // on large grids a longer list saves major passes and pivots (replayed
    // flow-update sequences: 20 k arcs best at 256, 327 k arcs at 2-4 k).
    std::vector<int> cand;

    bool run() {
        const int block = mcf_block > 0 ? mcf_block : std::max(16, (int)std::sqrt((double)na));
        const int kCand = std::min(4096, std::max(256, na / 128));
        cand.clear();
        int next = 0;
        const int64_t* cst = cost.data();
        const int* tl = tail.data();
        const int* hd = head.data();
        // the list lives in cl[0, nc); a block may overfill it by up to block - 1
        if ((int)cand.size() < kCand + block) cand.resize(kCand + block);
        int* cl = cand.data();
        int nc = 0;
        while (true) {
            int best = -1;
            int64_t best_rc = 0;
            for (int k = 0; k < nc;) {  // minor pass
                const int e = cl[k];
                const int64_t r = rc(e);
                if (r >= 0) {
                    cl[k] = cl[--nc];
                    continue;
                }
                if (r < best_rc) {
                    best_rc = r;
                    best = e;
                }
                ++k;
            }
            if (best < 0) {  // major pass
                nc = 0;
                const int64_t* pt = pot.data();
                int scanned = 0;
                while (scanned < na && nc < kCand) {
                    const int lim = std::min(block, na - scanned);
                    // arcs next, next + 1, ... (lim of them, wrapping at na): at most
                    // two contiguous ranges
                    int e = next, left = lim;
                    while (left > 0) {
                        const int stop = std::min(na, e + left);
                        left -= stop - e;
                        for (; e < stop; ++e) {
                            const int64_t r = cst[e] + pt[tl[e]] - pt[hd[e]];
                            if (r < 0) {
                                cl[nc++] = e;
                                if (r < best_rc) {
                                    best_rc = r;
                                    best = e;
                                }
                            }
                        }
                        if (e == na) e = 0;
                    }
                    next = e;
#ifdef MCF_STATS
                    st_scan += lim;
#endif
                    scanned += lim;
                }
                if (best < 0) return true;  // no arc of negative reduced cost: optimal
            }
            if (!pivot(best)) return false;
        }
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Solver with a persistent basis: the supplies (basic-cell masses) never change
// between flow updates, so the last optimal spanning tree and its flow stay a
// feasible, strongly feasible basis; a new solve only re-prices it with the new
// costs and pivots from there.
struct McfSolver {
    int n = 0;
    std::vector<int> arc_of;
    std::vector<int64_t> M;
    std::vector<double> m;
    NetworkSimplex ns;
};

static int check_input(int32_t n, const int32_t* nbr, const double* m) {
    if (n <= 0 || !nbr || !m) return DD_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!(m[i] > 0.0) || nbr[5 * i] != i) return DD_ERR_ARG;
        for (int k = 0; k < 5; ++k) {
            int j = nbr[5 * i + k];
            if (j < -1 || j >= n) return DD_ERR_ARG;
        }
    }
    return DD_OK;
}

int mcf_create(int32_t n, const int32_t* nbr, const double* m, McfSolver** out) {
    *out = nullptr;
    int rc = check_input(n, nbr, m);
    if (rc != DD_OK) return rc;
    McfSolver* S = new McfSolver();
    S->n = n;
    S->m.assign(m, m + n);
    NetworkSimplex& ns = S->ns;
    ns.nn = 2 * n;
    S->arc_of.assign(5 * (size_t)n, -1);
    S->M.resize(n);
    double msum = 0.0;
    for (int i = 0; i < n; ++i) msum += m[i];
    const double mscale = std::ldexp(1.0, 60) / msum;
    for (int i = 0; i < n; ++i) S->M[i] = std::max<int64_t>(1, (int64_t)std::llround(m[i] * mscale));
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 5; ++k) {
            int j = nbr[5 * i + k];
            if (j < 0) continue;
            S->arc_of[5 * i + k] = ns.na++;
            ns.tail.push_back(2 * i);  // source of cell i: node 2i, sink of cell j: node 2j + 1
            ns.head.push_back(2 * j + 1);
            ns.cost.push_back(0);
            ns.flow.push_back(k == 0 ? S->M[i] : 0);
        }
    const int nn = ns.nn;
    ns.parent.assign(nn, -1);
    ns.parc.assign(nn, -1);
    ns.pot.assign(nn, 0);
    // spanning tree of the cell grid by breadth-first search from cell 0, over
    // neighbour arcs; tree: s_root; t_i under s_p(i) (zero flow), s_i under t_i.
    std::vector<int> order;
    std::vector<char> seen(n, 0);
    order.reserve(n);
    order.push_back(0);
    seen[0] = 1;
    std::vector<int> via(n, -1), par_cell(n, -1);
    for (size_t h = 0; h < order.size(); ++h) {
        int p = order[h];
        for (int k = 1; k < 5; ++k) {
            int j = nbr[5 * p + k];
            if (j >= 0 && !seen[j]) {
                seen[j] = 1;
                par_cell[j] = p;
                via[j] = S->arc_of[5 * p + k];
                order.push_back(j);
            }
        }
    }
    if ((int)order.size() != n) {  // neighbourhood graph not connected
        delete S;
        return DD_ERR_ARG;
    }
    for (int idx = 0; idx < n; ++idx) {
        int i = order[idx];
        int self = S->arc_of[5 * i];
        int ti = 2 * i + 1, si = 2 * i;
        if (idx > 0) {
            int p = par_cell[i];
            ns.parent[ti] = 2 * p;
            ns.parc[ti] = via[i];
        }
        if (idx == 0) {  // root s_0; t_0 hangs below it
            ns.parent[ti] = si;
            ns.parc[ti] = self;
            ns.root = si;
        } else {
            ns.parent[si] = ti;
            ns.parc[si] = self;
        }
    }
    ns.build_thread();
    *out = S;
    return DD_OK;
}

int mcf_solve(McfSolver* S, const double* cbar, double* w, double* value, int32_t* pivots) {
    NetworkSimplex& ns = S->ns;
    const int n = S->n;
    double cmax = 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 5; ++k)
            if (S->arc_of[5 * i + k] >= 0) {
                if (!std::isfinite(cbar[5 * i + k])) return DD_ERR_ARG;
                cmax = std::max(cmax, std::fabs(cbar[5 * i + k]));
            }
    const double cscale = cmax > 0.0 ? std::ldexp(1.0, 40) / cmax : 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 5; ++k) {
            int a = S->arc_of[5 * i + k];
            if (a >= 0) ns.cost[a] = (int64_t)std::llround(cbar[5 * i + k] * cscale);
        }
    // re-price the current tree from its root
    ns.price_tree();
    const int64_t piv0 = ns.pivots;
    if (!ns.run()) return DD_ERR_FLOW;
    double val = 0.0;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 5; ++k) {
            int a = S->arc_of[5 * i + k];
            double wi = 0.0;
            if (a >= 0) {
                wi = S->m[i] * ((double)ns.flow[a] / (double)S->M[i]);
                val += wi * cbar[5 * i + k];
            }
            w[5 * i + k] = wi;
        }
    if (value) *value = val;
    if (pivots) *pivots = (int32_t)(ns.pivots - piv0);
    return DD_OK;
}

void mcf_destroy(McfSolver* S) { delete S; }

extern "C" int dd_min_cost_flow(int32_t n, const int32_t* nbr, const double* cbar, const double* m, double* w,
                                double* value, int32_t* pivots) {
    if (!cbar || !w) return DD_ERR_ARG;
    McfSolver* S = nullptr;
    int rc = mcf_create(n, nbr, m, &S);
    if (rc != DD_OK) return rc;
    rc = mcf_solve(S, cbar, w, value, pivots);
    mcf_destroy(S);
    return rc;
}
