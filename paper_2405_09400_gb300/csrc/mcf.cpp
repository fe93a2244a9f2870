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
//  * entering arcs by block search over the reduced costs;
//  * the tree is kept as parent pointers with doubly linked child lists; the
//    apex of a pivot cycle is found by marking the two upward walks; after a
//    pivot the cut subtree is re-rooted, and the potentials of the smaller of
//    the cut subtree and the rest are shifted (only differences matter).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/ddflow.h"

namespace {

int mcf_block = 0;  // entering-arc block size; 0 = sqrt(#arcs)

struct NetworkSimplex {
    int nn = 0;  // nodes: sources 0..n-1, sinks n..2n-1
    int na = 0;  // arcs
    std::vector<int> tail, head;
    std::vector<int64_t> cost, flow;
    std::vector<int> parent, parc, first_child, next_sib, prev_sib;
    std::vector<int64_t> pot;
    std::vector<int64_t> stamp;  // last pivot that visited the node (apex search)
    std::vector<int> pos;        // position of the node in its apex-search path
    std::vector<char> in_tree;
    std::vector<int> pu, pv, path, arcs, s1, s2, l1, l2;
    int64_t pivots = 0;
#ifdef MCF_STATS
    int64_t st_refresh = 0, st_path = 0, st_scan = 0, st_degenerate = 0;
#endif

    void add_child(int p, int c) {
        prev_sib[c] = -1;
        next_sib[c] = first_child[p];
        if (first_child[p] >= 0) prev_sib[first_child[p]] = c;
        first_child[p] = c;
    }
    void remove_child(int p, int c) {
        if (prev_sib[c] >= 0)
            next_sib[prev_sib[c]] = next_sib[c];
        else
            first_child[p] = next_sib[c];
        if (next_sib[c] >= 0) prev_sib[next_sib[c]] = prev_sib[c];
        next_sib[c] = prev_sib[c] = -1;
    }
    int64_t rc(int a) const { return cost[a] + pot[tail[a]] - pot[head[a]]; }

    // potentials of the whole tree from the root (node 0), tree arcs priced at 0
    void price_tree() {
        s1.clear();
        pot[0] = 0;
        for (int c = first_child[0]; c >= 0; c = next_sib[c]) s1.push_back(c);
        while (!s1.empty()) {
            int x = s1.back();
            s1.pop_back();
            int p = parent[x], a = parc[x];
            pot[x] = (tail[a] == p) ? pot[p] + cost[a] : pot[p] - cost[a];
            for (int c = first_child[x]; c >= 0; c = next_sib[c]) s1.push_back(c);
        }
    }

    bool pivot(int a) {
        const int u = tail[a], v = head[a];
        const int64_t tag = pivots + 1;
        // apex: walk up from u and v alternately, marking the nodes of each walk;
        // the first node reached that the other walk already marked is the apex.
        // pu / pv end up holding the nodes strictly below the apex on each side.
        pu.clear();
        pv.clear();
        stamp[u] = tag; pos[u] = 0; pu.push_back(u);
        stamp[v] = -tag; pos[v] = 0; pv.push_back(v);
        int x = u, y = v, apex = -1;
        while (apex < 0) {
            bool moved = false;
            if (parent[x] >= 0) {
                moved = true;
                x = parent[x];
                if (stamp[x] == -tag) { apex = x; pv.resize(pos[x]); break; }
                stamp[x] = tag; pos[x] = (int)pu.size(); pu.push_back(x);
            }
            if (parent[y] >= 0) {
                moved = true;
                y = parent[y];
                if (stamp[y] == tag) { apex = y; pu.resize(pos[y]); break; }
                stamp[y] = -tag; pos[y] = (int)pv.size(); pv.push_back(y);
            }
            if (!moved) return false;  // not a tree (cannot happen)
        }
        // backward arcs: on the u path (traversed apex -> u, downwards) arcs
        // pointing up; on the v path (traversed v -> apex, upwards) arcs pointing down.
        int64_t theta = INT64_MAX;
        for (int z : pu) {
            int e = parc[z];
            if (tail[e] == z) theta = std::min(theta, flow[e]);
        }
        for (int z : pv) {
            int e = parc[z];
            if (head[e] == z) theta = std::min(theta, flow[e]);
        }
        if (theta == INT64_MAX) return false;  // unbounded (cannot happen here)
#ifdef MCF_STATS
        st_path += pu.size() + pv.size();
        if (theta == 0) ++st_degenerate;
#endif
        // leaving arc: last blocking arc in the order apex->u, a, v->apex
        int leave_node = -1;
        bool on_v = false;
        for (int k = (int)pv.size() - 1; k >= 0; --k) {
            int z = pv[k], e = parc[z];
            if (head[e] == z && flow[e] == theta) { leave_node = z; on_v = true; break; }
        }
        if (leave_node < 0) {
            for (int k = 0; k < (int)pu.size(); ++k) {
                int z = pu[k], e = parc[z];
                if (tail[e] == z && flow[e] == theta) { leave_node = z; break; }
            }
        }
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
        // the subtree T_q below the leaving arc re-hangs at the endpoint r of a
        // inside it; its potentials shift by delta relative to the rest. Only
        // differences matter, so the smaller of T_q and the rest is shifted:
        // the two are enumerated in lockstep until one is exhausted.
        const int q = leave_node;
        const int r = on_v ? v : u;
        const int o = on_v ? u : v;
        const int64_t delta = on_v ? rc(a) : -rc(a);
        in_tree[parc[q]] = 0;
        in_tree[a] = 1;
        remove_child(parent[q], q);
        {
            s1.clear(); s2.clear(); l1.clear(); l2.clear();
            s1.push_back(q);
            s2.push_back(0);
            int done = 0;
            while (!done) {
                if (!s1.empty()) {
                    int z = s1.back(); s1.pop_back(); l1.push_back(z);
                    for (int c = first_child[z]; c >= 0; c = next_sib[c]) s1.push_back(c);
                } else done = 1;
                if (!done) {
                    if (!s2.empty()) {
                        int z = s2.back(); s2.pop_back(); l2.push_back(z);
                        for (int c = first_child[z]; c >= 0; c = next_sib[c]) s2.push_back(c);
                    } else done = 2;
                }
            }
            if (done == 1) {
                for (int z : l1) pot[z] += delta;
            } else {
                for (int z : l2) pot[z] -= delta;
            }
#ifdef MCF_STATS
            st_refresh += l1.size() + l2.size();
#endif
        }
        // path r -> q, reversed
        path.clear();
        for (int z = r; z != q; z = parent[z]) path.push_back(z);
        path.push_back(q);
        for (size_t t = 0; t + 1 < path.size(); ++t) remove_child(path[t + 1], path[t]);
        arcs.resize(path.size());
        for (size_t t = 0; t + 1 < path.size(); ++t) arcs[t] = parc[path[t]];
        for (size_t t = 0; t + 1 < path.size(); ++t) {
            int z0 = path[t], z1 = path[t + 1];
            parent[z1] = z0;
            parc[z1] = arcs[t];
            add_child(z0, z1);
        }
        parent[r] = o;
        parc[r] = a;
        add_child(o, r);
        ++pivots;
        return true;
    }

    bool run() {
        const int block = mcf_block > 0 ? mcf_block : std::max(16, (int)std::sqrt((double)na));
        int next = 0;
        while (true) {
            int best = -1;
            int64_t best_rc = 0;
            int scanned = 0;
            while (scanned < na) {
                int lim = std::min(block, na - scanned);
                for (int t = 0; t < lim; ++t) {
                    int e = next;
                    next = (next + 1 == na) ? 0 : next + 1;
                    if (in_tree[e]) continue;
#ifdef MCF_STATS
                    ++st_scan;
#endif
                    int64_t r = rc(e);
                    if (r < best_rc) { best_rc = r; best = e; }
                }
                scanned += lim;
                if (best >= 0) break;
            }
            if (best < 0) return true;
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
            ns.tail.push_back(i);
            ns.head.push_back(n + j);
            ns.cost.push_back(0);
            ns.flow.push_back(k == 0 ? S->M[i] : 0);
        }
    const int nn = ns.nn;
    ns.parent.assign(nn, -1);
    ns.parc.assign(nn, -1);
    ns.stamp.assign(nn, 0);
    ns.pos.assign(nn, 0);
    ns.first_child.assign(nn, -1);
    ns.next_sib.assign(nn, -1);
    ns.prev_sib.assign(nn, -1);
    ns.pot.assign(nn, 0);
    ns.in_tree.assign(ns.na, 0);
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
        int ti = n + i;
        if (idx > 0) {
            int p = par_cell[i];
            ns.parent[ti] = p;
            ns.parc[ti] = via[i];
            ns.in_tree[via[i]] = 1;
            ns.add_child(p, ti);
        }
        ns.in_tree[self] = 1;
        if (idx == 0) {  // root s_0; t_0 hangs below it
            ns.parent[ti] = i;
            ns.parc[ti] = self;
            ns.add_child(i, ti);
        } else {
            ns.parent[i] = ti;
            ns.parc[i] = self;
            ns.add_child(ti, i);
        }
    }
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
    // re-price the current tree from its root (node 0 = s_0 never has a parent)
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
