// Host-side graph generation and partitioning of libgnnmp.
//
// Sec. II-A of the paper: graph nodes are the GLL quadrature points of the hex
// elements of a spectral-element mesh, undirected edges join neighbouring
// quadrature points inside an element, and coincident nodes of neighbouring
// elements share one global id. On a conforming brick the union of the
// per-element 6-neighbour stencils is the 6-neighbour graph of the global GLL
// lattice, so the R=1 CSR is generated directly from lattice coordinates.
//
// Partitioning (Figs. 3-4): elements are assigned to R sub-graphs; sub-graph r
// keeps the nodes and stencil edges of its elements (local coincident nodes
// collapsed -- the "reduced" distributed graph). Edge degree d_ij (Eq. 5b) is
// the number of sub-graphs holding directed edge (i,j), node degree d_i
// (Eq. 8b) the number holding node i. The halo rows of Fig. 4 become, with all
// sub-graphs resident on one GPU, a copy list per shared global id.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "common.h"

namespace gnn {

namespace {
thread_local std::string g_last_error;
}

int set_error(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void clear_error() { g_last_error.clear(); }

const char* last_error() { return g_last_error.c_str(); }

// Gauss-Legendre-Lobatto points on [-1,1], ascending: the endpoints and the
// roots of P_p'. Newton iteration of von Winckel's "lglnodes" on
// x P_p(x) - P_{p-1}(x), started from the Chebyshev-Lobatto points.
static std::vector<double> gll_points(int p) {
    std::vector<double> x(p + 1);
    for (int k = 0; k <= p; ++k) x[k] = std::cos(M_PI * k / p);
    for (int it = 0; it < 100; ++it) {
        double change = 0.0;
        for (int k = 0; k <= p; ++k) {
            double pm1 = 1.0, pk = x[k];           // P_0, P_1
            for (int n = 2; n <= p; ++n) {
                double pn = ((2.0 * n - 1.0) * x[k] * pk - (n - 1.0) * pm1) / n;
                pm1 = pk;
                pk = pn;
            }
            // pk = P_p(x), pm1 = P_{p-1}(x)
            double dx = (x[k] * pk - pm1) / ((p + 1.0) * pk);
            x[k] -= dx;
            change = std::max(change, std::fabs(dx));
        }
        if (change < 1e-16) break;
    }
    std::sort(x.begin(), x.end());
    x[0] = -1.0;
    x[p] = 1.0;
    for (int k = 1; k < p; ++k) {            // exact antisymmetry
        if (k < p - k) {
            double m = 0.5 * (x[p - k] - x[k]);
            x[k] = -m;
            x[p - k] = m;
        } else if (k == p - k) {
            x[k] = 0.0;
        }
    }
    return x;
}

}  // namespace gnn

struct gnn_graph {
    int32_t kind = GNN_GRAPH_BRICK;
    int32_t nel[3] = {0, 0, 0};     // brick only
    int32_t p = 0;
    double extent[3] = {0, 0, 0};
    int32_t periodic[3] = {0, 0, 0};
    int32_t L[3] = {0, 0, 0};
    int64_t n_nodes = 0;
    int64_t n_elem = 0;
    std::vector<double> pos;        // [N*3]
    std::vector<int64_t> row_ptr;   // [N+1]
    std::vector<int64_t> col;       // [E]
    // element meshes (GNN_GRAPH_ELEMENTS)
    std::vector<int64_t> elem_ptr, elem_nodes, edge_ptr;
    std::vector<int32_t> edge_pairs;
    std::vector<double> centre;     // [n_elem*3] mean node position
};

struct gnn_partition {
    int32_t R;
    int32_t max_in_degree;
    int32_t tile_edges;     // edge cap of the current tiles
    std::vector<int64_t> row_offsets, edge_offsets;
    std::vector<int64_t> row_gid;
    std::vector<int32_t> row_ptr, col;
    std::vector<uint8_t> edge_deg, node_deg;
    std::vector<int32_t> t_ptr, t_eid;
    std::vector<int32_t> halo_ptr, halo_rows;
    std::vector<int32_t> edge_tiles;
    std::vector<uint8_t> tile_meta;
    std::vector<double> row_pos;
    std::vector<int64_t> part_stats;
};

namespace {

using gnn::set_error;

struct Lattice {
    int32_t nel[3], L[3], p;
    int32_t periodic[3];
    int64_t gid(int64_t ix, int64_t iy, int64_t iz) const { return ix + L[0] * (iy + (int64_t)L[1] * iz); }
    void coords(int64_t g, int64_t c[3]) const {
        c[0] = g % L[0];
        c[1] = (g / L[0]) % L[1];
        c[2] = g / ((int64_t)L[0] * L[1]);
    }
    // element indices along one axis that contain lattice index i; returns count (1 or 2)
    int elems_of_point(int a, int64_t i, int64_t out[2]) const {
        int n = 0;
        int64_t e = i / p;
        if (i % p == 0) {
            int64_t left = e - 1;
            if (periodic[a]) left = (left + nel[a]) % nel[a];
            if (left >= 0) out[n++] = left;
            if (e < nel[a]) out[n++] = e;
        } else {
            out[n++] = e;
        }
        return n;
    }
    int64_t elem_id(int64_t ex, int64_t ey, int64_t ez) const { return ex + nel[0] * (ey + (int64_t)nel[1] * ez); }
};

Lattice lattice_of(const gnn_graph* g) {
    Lattice lt;
    for (int a = 0; a < 3; ++a) {
        lt.nel[a] = g->nel[a];
        lt.L[a] = g->L[a];
        lt.periodic[a] = g->periodic[a];
    }
    lt.p = g->p;
    return lt;
}

template <class F>
void parallel_for(int64_t n, F f) {
    unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
    if (n < 2 || nt == 1) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next(0);
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt && (int64_t)t < n; ++t)
        th.emplace_back([&] {
            for (int64_t i; (i = next.fetch_add(1)) < n;) f(i);
        });
    for (auto& t : th) t.join();
}

// Element -> part by recursive coordinate bisection of element centres.
void rcb_split(const std::vector<double>& centre, std::vector<int64_t>& elems, int64_t lo, int64_t hi,
               int32_t r0, int32_t nr, const std::vector<double>& w, std::vector<int32_t>& part) {
    if (nr == 1) {
        for (int64_t i = lo; i < hi; ++i) part[elems[i]] = r0;
        return;
    }
    int axis = 0;
    double ext[3];
    for (int a = 0; a < 3; ++a) {
        double mn = std::numeric_limits<double>::infinity(), mx = -mn;
        for (int64_t i = lo; i < hi; ++i) {
            double c = centre[elems[i] * 3 + a];
            mn = std::min(mn, c);
            mx = std::max(mx, c);
        }
        ext[a] = mx - mn;
    }
    for (int a = 1; a < 3; ++a)
        if (ext[a] > ext[axis]) axis = a;
    std::sort(elems.begin() + lo, elems.begin() + hi, [&](int64_t u, int64_t v) {
        double cu = centre[u * 3 + axis], cv = centre[v * 3 + axis];
        if (cu != cv) return cu < cv;
        return u < v;
    });
    int32_t nl = nr / 2;
    double wl = 0.0, wr = 0.0;
    for (int32_t k = r0; k < r0 + nl; ++k) wl += w[k];
    for (int32_t k = r0 + nl; k < r0 + nr; ++k) wr += w[k];
    int64_t n = hi - lo;
    int64_t cut = (int64_t)std::floor((double)n * wl / (wl + wr) + 0.5);
    cut = std::min(std::max(cut, (int64_t)nl), n - (nr - nl));
    rcb_split(centre, elems, lo, lo + cut, r0, nl, w, part);
    rcb_split(centre, elems, lo + cut, hi, r0 + nl, nr - nl, w, part);
}

}  // namespace

extern "C" {

const char* gnn_last_error(void) { return gnn::last_error(); }

int gnn_version(void) { return 1 * 10000 + 0 * 100 + 0; }

int gnn_graph_build(const gnn_mesh_desc* d, gnn_graph** out) {
    GNN_REQUIRE(d && out, GNN_EINVAL, "gnn_graph_build: NULL argument");
    *out = nullptr;
    GNN_REQUIRE(d->p >= 1 && d->p <= 15, GNN_EINVAL, "gnn_graph_build: p=%d out of range 1..15", d->p);
    for (int a = 0; a < 3; ++a) {
        GNN_REQUIRE(d->nel[a] >= 1, GNN_EINVAL, "gnn_graph_build: nel[%d]=%d < 1", a, d->nel[a]);
        GNN_REQUIRE(d->extent[a] > 0.0, GNN_EINVAL, "gnn_graph_build: extent[%d] <= 0", a);
        GNN_REQUIRE(!d->periodic[a] || (int64_t)d->nel[a] * d->p >= 3, GNN_EINVAL,
                    "gnn_graph_build: periodic axis %d needs nel*p >= 3", a);
    }
    GNN_REQUIRE(d->jitter_frac >= 0.0 && d->jitter_frac < 0.5, GNN_EINVAL,
                "gnn_graph_build: jitter_frac must be in [0, 0.5)");
    gnn_graph* g = new (std::nothrow) gnn_graph();
    GNN_REQUIRE(g, GNN_ENOMEM, "gnn_graph_build: out of host memory");
    try {
        g->kind = GNN_GRAPH_BRICK;
        g->p = d->p;
        g->n_elem = (int64_t)d->nel[0] * d->nel[1] * d->nel[2];
        int64_t N = 1;
        for (int a = 0; a < 3; ++a) {
            g->nel[a] = d->nel[a];
            g->extent[a] = d->extent[a];
            g->periodic[a] = d->periodic[a] ? 1 : 0;
            g->L[a] = d->nel[a] * d->p + (g->periodic[a] ? 0 : 1);
            N *= g->L[a];
        }
        GNN_REQUIRE(N * 6 < (int64_t)std::numeric_limits<int32_t>::max() * 4, GNN_ESHAPE,
                    "gnn_graph_build: graph too large");
        g->n_nodes = N;
        const int p = d->p;
        std::vector<double> xi = gnn::gll_points(p);
        std::vector<double> coord[3], spacing[3];
        for (int a = 0; a < 3; ++a) {
            int La = g->L[a];
            double h = d->extent[a] / d->nel[a];
            coord[a].assign(La, 0.0);
            for (int e = 0; e < d->nel[a]; ++e)
                for (int k = 0; k <= p; ++k) {
                    int gi = e * p + k;
                    if (gi < La) coord[a][gi] = (e + 0.5 * (xi[k] + 1.0)) * h;
                }
            spacing[a].assign(La, std::numeric_limits<double>::infinity());
            for (int i = 0; i < La; ++i) {
                double s = spacing[a][i];
                if (i > 0) s = std::min(s, coord[a][i] - coord[a][i - 1]);
                if (i + 1 < La) s = std::min(s, coord[a][i + 1] - coord[a][i]);
                if (g->periodic[a] && (i == 0 || i == La - 1))
                    s = std::min(s, coord[a][0] + d->extent[a] - coord[a][La - 1]);
                spacing[a][i] = s;
            }
        }
        g->pos.resize(N * 3);
        Lattice lt = lattice_of(g);
        parallel_for((N + 65535) / 65536, [&](int64_t blk) {
            int64_t g0 = blk * 65536, g1 = std::min(N, g0 + 65536);
            for (int64_t gi = g0; gi < g1; ++gi) {
                int64_t c[3];
                lt.coords(gi, c);
                for (int a = 0; a < 3; ++a) {
                    double v = coord[a][c[a]];
                    if (d->jitter && d->jitter_frac != 0.0) {
                        bool face = !g->periodic[a] && (c[a] == 0 || c[a] == g->L[a] - 1);
                        if (!face) v = v + d->jitter[gi * 3 + a] * d->jitter_frac * spacing[a][c[a]];
                    }
                    g->pos[gi * 3 + a] = v;
                }
            }
        });
        // lattice CSR: every lattice-adjacent pair lies in a common element
        g->row_ptr.resize(N + 1);
        g->row_ptr[0] = 0;
        std::vector<uint8_t> deg(N);
        parallel_for((N + 65535) / 65536, [&](int64_t blk) {
            int64_t g0 = blk * 65536, g1 = std::min(N, g0 + 65536);
            for (int64_t gi = g0; gi < g1; ++gi) {
                int64_t c[3];
                lt.coords(gi, c);
                int n = 0;
                for (int a = 0; a < 3; ++a) {
                    if (g->periodic[a]) n += 2;
                    else n += (c[a] > 0) + (c[a] < g->L[a] - 1);
                }
                deg[gi] = (uint8_t)n;
            }
        });
        for (int64_t gi = 0; gi < N; ++gi) g->row_ptr[gi + 1] = g->row_ptr[gi] + deg[gi];
        g->col.resize(g->row_ptr[N]);
        parallel_for((N + 65535) / 65536, [&](int64_t blk) {
            int64_t g0 = blk * 65536, g1 = std::min(N, g0 + 65536);
            for (int64_t gi = g0; gi < g1; ++gi) {
                int64_t c[3];
                lt.coords(gi, c);
                int64_t nb[6];
                int n = 0;
                for (int a = 0; a < 3; ++a)
                    for (int s = -1; s <= 1; s += 2) {
                        int64_t cc[3] = {c[0], c[1], c[2]};
                        cc[a] += s;
                        if (cc[a] < 0 || cc[a] >= g->L[a]) {
                            if (!g->periodic[a]) continue;
                            cc[a] = (cc[a] + g->L[a]) % g->L[a];
                        }
                        nb[n++] = lt.gid(cc[0], cc[1], cc[2]);
                    }
                std::sort(nb, nb + n);
                std::copy(nb, nb + n, g->col.begin() + g->row_ptr[gi]);
            }
        });
    } catch (const std::bad_alloc&) {
        delete g;
        return set_error(GNN_ENOMEM, "gnn_graph_build: out of host memory");
    }
    *out = g;
    gnn::clear_error();
    return GNN_OK;
}

int gnn_graph_build_elements(const gnn_elem_mesh_desc* d, gnn_graph** out) {
    GNN_REQUIRE(d && out, GNN_EINVAL, "gnn_graph_build_elements: NULL argument");
    *out = nullptr;
    const int64_t N = d->n_nodes, ne = d->n_elem;
    GNN_REQUIRE(N >= 1 && ne >= 1, GNN_EINVAL, "gnn_graph_build_elements: needs a node and an element");
    GNN_REQUIRE(N < (int64_t)std::numeric_limits<int32_t>::max(), GNN_ESHAPE,
                "gnn_graph_build_elements: more than 2^31-1 nodes");
    GNN_REQUIRE(d->pos && d->elem_ptr && d->edge_ptr, GNN_EINVAL, "gnn_graph_build_elements: NULL array");
    GNN_REQUIRE(d->elem_ptr[0] == 0 && d->edge_ptr[0] == 0, GNN_EINVAL,
                "gnn_graph_build_elements: offsets must start at 0");
    for (int64_t e = 0; e < ne; ++e) {
        GNN_REQUIRE(d->elem_ptr[e + 1] > d->elem_ptr[e], GNN_EINVAL,
                    "gnn_graph_build_elements: element %lld has no node", (long long)e);
        GNN_REQUIRE(d->edge_ptr[e + 1] >= d->edge_ptr[e], GNN_EINVAL,
                    "gnn_graph_build_elements: edge offsets descend at element %lld", (long long)e);
    }
    const int64_t n_en = d->elem_ptr[ne], n_pairs = d->edge_ptr[ne];
    GNN_REQUIRE(d->elem_nodes, GNN_EINVAL, "gnn_graph_build_elements: NULL elem_nodes");
    GNN_REQUIRE(n_pairs == 0 || d->edge_pairs, GNN_EINVAL, "gnn_graph_build_elements: NULL edge_pairs");
    std::vector<uint8_t> covered;
    gnn_graph* g = new (std::nothrow) gnn_graph();
    GNN_REQUIRE(g, GNN_ENOMEM, "gnn_graph_build_elements: out of host memory");
    try {
        covered.assign(N, 0);
        for (int64_t e = 0; e < ne; ++e) {
            const int64_t k0 = d->elem_ptr[e], nk = d->elem_ptr[e + 1] - k0;
            for (int64_t k = k0; k < k0 + nk; ++k) {
                const int64_t id = d->elem_nodes[k];
                if (id < 0 || id >= N) {
                    delete g;
                    return set_error(GNN_EINVAL, "gnn_graph_build_elements: element %lld node id %lld out of range",
                                     (long long)e, (long long)id);
                }
                covered[id] |= 1;
            }
            for (int64_t k = d->edge_ptr[e]; k < d->edge_ptr[e + 1]; ++k) {
                const int32_t u = d->edge_pairs[2 * k], v = d->edge_pairs[2 * k + 1];
                if (u < 0 || v < 0 || u >= nk || v >= nk || d->elem_nodes[k0 + u] == d->elem_nodes[k0 + v]) {
                    delete g;
                    return set_error(GNN_EINVAL, "gnn_graph_build_elements: element %lld pair %lld (%d, %d) invalid",
                                     (long long)e, (long long)(k - d->edge_ptr[e]), u, v);
                }
                covered[d->elem_nodes[k0 + u]] |= 2;
                covered[d->elem_nodes[k0 + v]] |= 2;
            }
        }
        for (int64_t i = 0; i < N; ++i)
            if (covered[i] != 3) {
                delete g;
                return set_error(GNN_EINVAL, "gnn_graph_build_elements: node %lld is in no %s", (long long)i,
                                 covered[i] ? "edge" : "element");
            }
        g->kind = GNN_GRAPH_ELEMENTS;
        g->n_nodes = N;
        g->n_elem = ne;
        g->pos.assign(d->pos, d->pos + N * 3);
        g->elem_ptr.assign(d->elem_ptr, d->elem_ptr + ne + 1);
        g->elem_nodes.assign(d->elem_nodes, d->elem_nodes + n_en);
        g->edge_ptr.assign(d->edge_ptr, d->edge_ptr + ne + 1);
        g->edge_pairs.assign(d->edge_pairs, d->edge_pairs + 2 * n_pairs);
        g->centre.assign(ne * 3, 0.0);
        for (int64_t e = 0; e < ne; ++e) {
            const int64_t k0 = d->elem_ptr[e], k1 = d->elem_ptr[e + 1];
            for (int a = 0; a < 3; ++a) {
                double c = 0.0;
                for (int64_t k = k0; k < k1; ++k) c += g->pos[d->elem_nodes[k] * 3 + a];
                g->centre[e * 3 + a] = c / (double)(k1 - k0);
            }
        }
        // R=1 graph: union of the element edges, both directions, receiver-sorted
        std::vector<int64_t> keys;
        keys.reserve(2 * n_pairs);
        for (int64_t e = 0; e < ne; ++e) {
            const int64_t* en = d->elem_nodes + d->elem_ptr[e];
            for (int64_t k = d->edge_ptr[e]; k < d->edge_ptr[e + 1]; ++k) {
                const int64_t u = en[d->edge_pairs[2 * k]], v = en[d->edge_pairs[2 * k + 1]];
                keys.push_back(u * N + v);
                keys.push_back(v * N + u);
            }
        }
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        g->row_ptr.assign(N + 1, 0);
        g->col.resize(keys.size());
        for (size_t t = 0; t < keys.size(); ++t) {
            g->row_ptr[keys[t] / N + 1]++;
            g->col[t] = keys[t] % N;
        }
        for (int64_t i = 0; i < N; ++i) g->row_ptr[i + 1] += g->row_ptr[i];
    } catch (const std::bad_alloc&) {
        delete g;
        return set_error(GNN_ENOMEM, "gnn_graph_build_elements: out of host memory");
    }
    *out = g;
    gnn::clear_error();
    return GNN_OK;
}

void gnn_graph_destroy(gnn_graph* g) { delete g; }

int gnn_graph_get_info(const gnn_graph* g, gnn_graph_info* info) {
    GNN_REQUIRE(g && info, GNN_EINVAL, "gnn_graph_get_info: NULL argument");
    info->n_nodes = g->n_nodes;
    info->n_edges = (int64_t)g->col.size();
    info->n_elem = g->n_elem;
    for (int a = 0; a < 3; ++a) info->L[a] = g->L[a];
    info->p = g->p;
    info->n_elem_nodes = g->kind == GNN_GRAPH_BRICK ? g->n_elem * (g->p + 1) * (g->p + 1) * (g->p + 1)
                                                    : (int64_t)g->elem_nodes.size();
    info->kind = g->kind;
    int64_t md = 0;
    for (int64_t i = 0; i < g->n_nodes; ++i) md = std::max(md, g->row_ptr[i + 1] - g->row_ptr[i]);
    info->max_degree = (int32_t)md;
    return GNN_OK;
}

int gnn_graph_copy_pos(const gnn_graph* g, double* pos) {
    GNN_REQUIRE(g && pos, GNN_EINVAL, "gnn_graph_copy_pos: NULL argument");
    std::memcpy(pos, g->pos.data(), g->pos.size() * sizeof(double));
    return GNN_OK;
}

int gnn_graph_copy_csr(const gnn_graph* g, int64_t* row_ptr, int64_t* col) {
    GNN_REQUIRE(g && row_ptr && col, GNN_EINVAL, "gnn_graph_copy_csr: NULL argument");
    std::memcpy(row_ptr, g->row_ptr.data(), g->row_ptr.size() * sizeof(int64_t));
    std::memcpy(col, g->col.data(), g->col.size() * sizeof(int64_t));
    return GNN_OK;
}

int gnn_graph_copy_elements(const gnn_graph* g, int64_t* en) {
    GNN_REQUIRE(g && en, GNN_EINVAL, "gnn_graph_copy_elements: NULL argument");
    if (g->kind == GNN_GRAPH_ELEMENTS) {
        std::memcpy(en, g->elem_nodes.data(), g->elem_nodes.size() * sizeof(int64_t));
        return GNN_OK;
    }
    Lattice lt = lattice_of(g);
    const int q = g->p + 1;
    int64_t n_elem = (int64_t)g->nel[0] * g->nel[1] * g->nel[2];
    for (int64_t e = 0; e < n_elem; ++e) {
        int64_t ex = e % g->nel[0], ey = (e / g->nel[0]) % g->nel[1], ez = e / ((int64_t)g->nel[0] * g->nel[1]);
        for (int k = 0; k < q; ++k)
            for (int j = 0; j < q; ++j)
                for (int i = 0; i < q; ++i)
                    en[e * q * q * q + i + q * (j + q * k)] =
                        lt.gid((ex * g->p + i) % g->L[0], (ey * g->p + j) % g->L[1], (ez * g->p + k) % g->L[2]);
    }
    return GNN_OK;
}

int gnn_graph_copy_element_ptr(const gnn_graph* g, int64_t* ptr) {
    GNN_REQUIRE(g && ptr, GNN_EINVAL, "gnn_graph_copy_element_ptr: NULL argument");
    if (g->kind == GNN_GRAPH_ELEMENTS) {
        std::memcpy(ptr, g->elem_ptr.data(), g->elem_ptr.size() * sizeof(int64_t));
        return GNN_OK;
    }
    const int64_t q3 = (int64_t)(g->p + 1) * (g->p + 1) * (g->p + 1);
    for (int64_t e = 0; e <= g->n_elem; ++e) ptr[e] = e * q3;
    return GNN_OK;
}

// Receiver-aligned edge tiles: consecutive rows, at most `cap` edges and at
// most GNN_EDGE_TILE rows per tile (a row's edges never straddle two tiles),
// and one fixed-size record per tile (layout in gnnmp.h, GNN_P_TILE_META).
static void build_edge_tiles(gnn_partition* P, int32_t cap) {
    const int64_t NR = (int64_t)P->row_ptr.size() - 1;
    P->tile_edges = cap;
    P->edge_tiles.clear();
    P->edge_tiles.push_back(0);
    int64_t r0 = 0;
    while (r0 < NR) {
        int64_t r1 = r0;
        while (r1 < NR && r1 - r0 < GNN_EDGE_TILE && P->row_ptr[r1 + 1] - P->row_ptr[r0] <= cap) ++r1;
        P->edge_tiles.push_back((int32_t)r1);
        r0 = r1;
    }
    const int64_t nt = (int64_t)P->edge_tiles.size() - 1;
    P->tile_meta.assign((size_t)nt * GNN_TILE_META_BYTES, 0);
    parallel_for(nt, [&](int64_t t) {
        uint8_t* rec = P->tile_meta.data() + (size_t)t * GNN_TILE_META_BYTES;
        int32_t* hdr = reinterpret_cast<int32_t*>(rec);
        int32_t* rp = reinterpret_cast<int32_t*>(rec + 16);
        int16_t* seg = reinterpret_cast<int16_t*>(rec + 544);
        int32_t* cl = reinterpret_cast<int32_t*>(rec + 800);
        float* w = reinterpret_cast<float*>(rec + 1312);
        const int32_t r0 = P->edge_tiles[t], r1 = P->edge_tiles[t + 1];
        const int32_t e0 = P->row_ptr[r0], ne = P->row_ptr[r1] - e0;
        hdr[0] = r0;
        hdr[1] = r1;
        hdr[2] = e0;
        hdr[3] = ne;
        for (int32_t i = 0; i <= r1 - r0; ++i) rp[i] = P->row_ptr[r0 + i] - e0;
        for (int32_t i = 0; i < r1 - r0; ++i)
            for (int32_t e = rp[i]; e < rp[i + 1]; ++e) seg[e] = (int16_t)i;
        for (int32_t e = 0; e < ne; ++e) {
            cl[e] = P->col[e0 + e];
            w[e] = 1.0f / (float)P->edge_deg[e0 + e];
        }
    });
}

}  // extern "C"

namespace {

// Reduced sub-graphs before concatenation: sub-graph r holds the global ids
// nodes[r] (ascending) and a receiver CSR over them (lcol = local sender row,
// senders ascending), with d_ij per edge and d_i per row.
struct LocalGraphs {
    std::vector<std::vector<int64_t>> nodes;
    std::vector<std::vector<int32_t>> lptr, lcol, ldeg, ndeg;
    void reset(int32_t R) {
        nodes.assign(R, {});
        lptr.assign(R, {});
        lcol.assign(R, {});
        ldeg.assign(R, {});
        ndeg.assign(R, {});
    }
};

// Brick: nodes, stencil edges and their multiplicities from lattice coordinates.
int local_graphs_brick(const gnn_graph* g, int32_t R, const std::vector<int32_t>& part, LocalGraphs& LG) {
    Lattice lt = lattice_of(g);
    const int p = g->p;
    const int q = p + 1;
    const int64_t n_elem = g->n_elem;
    // parts holding a lattice point / a lattice edge
    auto node_parts = [&](int64_t gi, int32_t* ps) {
        int64_t c[3], ea[3][2];
        int na[3];
        lt.coords(gi, c);
        for (int a = 0; a < 3; ++a) na[a] = lt.elems_of_point(a, c[a], ea[a]);
        int n = 0;
        for (int i = 0; i < na[0]; ++i)
            for (int j = 0; j < na[1]; ++j)
                for (int k = 0; k < na[2]; ++k) {
                    int32_t r = part[lt.elem_id(ea[0][i], ea[1][j], ea[2][k])];
                    bool seen = false;
                    for (int t = 0; t < n; ++t) seen |= (ps[t] == r);
                    if (!seen) ps[n++] = r;
                }
        return n;
    };
    auto edge_parts = [&](int64_t gu, int64_t gv, int32_t* ps) {
        int64_t cu[3], cv[3];
        lt.coords(gu, cu);
        lt.coords(gv, cv);
        int axis = 0;
        for (int a = 0; a < 3; ++a)
            if (cu[a] != cv[a]) axis = a;
        int64_t ea[3][2];
        int na[3];
        for (int a = 0; a < 3; ++a) {
            if (a == axis) {
                int64_t lo = cu[a], hi = cv[a];
                // segment index = lower end, or the wrap segment L-1 -> 0
                int64_t seg = (std::llabs(hi - lo) == 1) ? std::min(lo, hi) : std::max(lo, hi);
                ea[a][0] = seg / p;
                na[a] = 1;
            } else {
                na[a] = lt.elems_of_point(a, cu[a], ea[a]);
            }
        }
        int n = 0;
        for (int i = 0; i < na[0]; ++i)
            for (int j = 0; j < na[1]; ++j)
                for (int k = 0; k < na[2]; ++k) {
                    int32_t r = part[lt.elem_id(ea[0][i], ea[1][j], ea[2][k])];
                    bool seen = false;
                    for (int t = 0; t < n; ++t) seen |= (ps[t] == r);
                    if (!seen) ps[n++] = r;
                }
        return n;
    };
    LG.reset(R);
    std::vector<std::vector<int64_t>> elems_of(R);
    for (int64_t e = 0; e < n_elem; ++e) elems_of[part[e]].push_back(e);
    std::atomic<int> err(0);
    parallel_for(R, [&](int64_t r) {
        std::vector<int64_t>& nd = LG.nodes[r];
        nd.reserve(elems_of[r].size() * q * q * q);
        for (int64_t e : elems_of[r]) {
            int64_t ex = e % g->nel[0], ey = (e / g->nel[0]) % g->nel[1], ez = e / ((int64_t)g->nel[0] * g->nel[1]);
            for (int k = 0; k < q; ++k)
                for (int j = 0; j < q; ++j)
                    for (int i = 0; i < q; ++i)
                        nd.push_back(lt.gid((ex * p + i) % g->L[0], (ey * p + j) % g->L[1], (ez * p + k) % g->L[2]));
        }
        std::sort(nd.begin(), nd.end());
        nd.erase(std::unique(nd.begin(), nd.end()), nd.end());
        const int64_t n = (int64_t)nd.size();
        LG.lptr[r].assign(n + 1, 0);
        LG.ndeg[r].resize(n);
        int32_t ps[8];
        for (int64_t i = 0; i < n; ++i) {
            int64_t gi = nd[i];
            LG.ndeg[r][i] = node_parts(gi, ps);
            for (int64_t t = g->row_ptr[gi]; t < g->row_ptr[gi + 1]; ++t) {
                int64_t gj = g->col[t];
                int m = edge_parts(gi, gj, ps);
                bool mine = false;
                for (int s = 0; s < m; ++s) mine |= (ps[s] == (int32_t)r);
                if (!mine) continue;
                auto it = std::lower_bound(nd.begin(), nd.end(), gj);
                if (it == nd.end() || *it != gj) {
                    err = 1;
                    continue;
                }
                LG.lcol[r].push_back((int32_t)(it - nd.begin()));
                LG.ldeg[r].push_back(m);
            }
            LG.lptr[r][i + 1] = (int32_t)LG.lcol[r].size();
        }
    });
    GNN_REQUIRE(!err, GNN_EHALO, "gnn_partition: internal edge/node mismatch");
    return GNN_OK;
}

// Element mesh: sub-graph r keeps the nodes and the edges (both directions) of
// its elements; d_ij and d_i count the sub-graphs holding each edge and node.
int local_graphs_elements(const gnn_graph* g, int32_t R, const std::vector<int32_t>& part, LocalGraphs& LG) {
    const int64_t N = g->n_nodes, n_elem = g->n_elem;
    LG.reset(R);
    std::vector<std::vector<int64_t>> elems_of(R), keys(R);
    for (int64_t e = 0; e < n_elem; ++e) elems_of[part[e]].push_back(e);
    parallel_for(R, [&](int64_t r) {
        std::vector<int64_t>& nd = LG.nodes[r];
        std::vector<int64_t>& ky = keys[r];
        for (int64_t e : elems_of[r]) {
            const int64_t* en = g->elem_nodes.data() + g->elem_ptr[e];
            nd.insert(nd.end(), en, en + (g->elem_ptr[e + 1] - g->elem_ptr[e]));
            for (int64_t k = g->edge_ptr[e]; k < g->edge_ptr[e + 1]; ++k) {
                const int64_t u = en[g->edge_pairs[2 * k]], v = en[g->edge_pairs[2 * k + 1]];
                ky.push_back(u * N + v);
                ky.push_back(v * N + u);
            }
        }
        std::sort(nd.begin(), nd.end());
        nd.erase(std::unique(nd.begin(), nd.end()), nd.end());
        std::sort(ky.begin(), ky.end());
        ky.erase(std::unique(ky.begin(), ky.end()), ky.end());
    });
    std::vector<int32_t> ncount(N, 0);
    for (int32_t r = 0; r < R; ++r)
        for (int64_t gi : LG.nodes[r]) ncount[gi]++;
    std::vector<int64_t> all;
    {
        size_t tot = 0;
        for (int32_t r = 0; r < R; ++r) tot += keys[r].size();
        all.reserve(tot);
        for (int32_t r = 0; r < R; ++r) all.insert(all.end(), keys[r].begin(), keys[r].end());
    }
    std::sort(all.begin(), all.end());
    std::vector<int64_t> uk;
    std::vector<int32_t> uc;
    for (size_t t = 0; t < all.size();) {
        size_t u = t;
        while (u < all.size() && all[u] == all[t]) ++u;
        uk.push_back(all[t]);
        uc.push_back((int32_t)(u - t));
        t = u;
    }
    std::vector<int64_t>().swap(all);
    parallel_for(R, [&](int64_t r) {
        const std::vector<int64_t>& nd = LG.nodes[r];
        const int64_t n = (int64_t)nd.size();
        LG.lptr[r].assign(n + 1, 0);
        LG.ndeg[r].resize(n);
        for (int64_t i = 0; i < n; ++i) LG.ndeg[r][i] = ncount[nd[i]];
        LG.lcol[r].resize(keys[r].size());
        LG.ldeg[r].resize(keys[r].size());
        for (size_t t = 0; t < keys[r].size(); ++t) {
            const int64_t key = keys[r][t];
            const int64_t ri = std::lower_bound(nd.begin(), nd.end(), key / N) - nd.begin();
            LG.lptr[r][ri + 1]++;
            LG.lcol[r][t] = (int32_t)(std::lower_bound(nd.begin(), nd.end(), key % N) - nd.begin());
            LG.ldeg[r][t] = uc[std::lower_bound(uk.begin(), uk.end(), key) - uk.begin()];
        }
        for (int64_t i = 0; i < n; ++i) LG.lptr[r][i + 1] += LG.lptr[r][i];
    });
    return GNN_OK;
}

// A row of in-degree > cap becomes k = ceil(degree / cap) consecutive copies:
// copy c receives the c-th of k near-equal consecutive runs of the row's
// in-edges and is the sender of the edges back to that run's nodes. d_i then
// counts every row holding the node.
int split_hubs(LocalGraphs& LG, int32_t R, int32_t cap) {
    std::vector<std::vector<std::pair<int64_t, int32_t>>> extra(R);
    parallel_for(R, [&](int64_t r) {
        const std::vector<int64_t>& nd = LG.nodes[r];
        const std::vector<int32_t>& lp = LG.lptr[r];
        const std::vector<int32_t>& lc = LG.lcol[r];
        const int64_t n = (int64_t)nd.size();
        std::vector<int32_t> k(n);
        bool any = false;
        for (int64_t i = 0; i < n; ++i) {
            const int32_t deg = lp[i + 1] - lp[i];
            k[i] = deg > cap ? (deg + cap - 1) / cap : 1;
            any |= k[i] > 1;
        }
        if (!any) return;
        auto run_start = [&](int64_t i, int32_t c) {
            return lp[i] + (int32_t)((int64_t)c * (lp[i + 1] - lp[i]) / k[i]);
        };
        std::vector<int32_t> first(n + 1, 0);
        for (int64_t i = 0; i < n; ++i) first[i + 1] = first[i] + k[i];
        std::vector<int64_t> nd2(first[n]);
        std::vector<int32_t> lp2(first[n] + 1), lc2(lc.size()), ndeg2(first[n]);
        for (int64_t i = 0; i < n; ++i) {
            for (int32_t c = 0; c < k[i]; ++c) {
                nd2[first[i] + c] = nd[i];
                ndeg2[first[i] + c] = LG.ndeg[r][i];
                lp2[first[i] + c] = run_start(i, c);
            }
            if (k[i] > 1) extra[r].emplace_back(nd[i], k[i] - 1);
        }
        lp2[first[n]] = lp[n];
        for (int64_t i = 0; i < n; ++i)
            for (int32_t t = lp[i]; t < lp[i + 1]; ++t) {
                const int32_t j = lc[t];
                int32_t c = 0;
                if (k[j] > 1) {
                    auto b = lc.begin() + lp[j], e = lc.begin() + lp[j + 1];
                    auto it = std::lower_bound(b, e, (int32_t)i);
                    if (it != e && *it == (int32_t)i) {
                        const int32_t pos = (int32_t)(it - lc.begin());
                        c = k[j] - 1;
                        while (run_start(j, c) > pos) --c;
                    }
                }
                lc2[t] = first[j] + c;
            }
        LG.nodes[r].swap(nd2);
        LG.lptr[r].swap(lp2);
        LG.lcol[r].swap(lc2);
        LG.ndeg[r].swap(ndeg2);
    });
    std::vector<std::pair<int64_t, int32_t>> add;
    for (int32_t r = 0; r < R; ++r) add.insert(add.end(), extra[r].begin(), extra[r].end());
    if (add.empty()) return GNN_OK;
    std::sort(add.begin(), add.end());
    std::vector<std::pair<int64_t, int32_t>> tot;
    for (auto& a : add) {
        if (!tot.empty() && tot.back().first == a.first) tot.back().second += a.second;
        else tot.push_back(a);
    }
    parallel_for(R, [&](int64_t r) {
        for (size_t i = 0; i < LG.nodes[r].size(); ++i) {
            auto it = std::lower_bound(tot.begin(), tot.end(), std::make_pair(LG.nodes[r][i], (int32_t)-1));
            if (it != tot.end() && it->first == LG.nodes[r][i]) LG.ndeg[r][i] += it->second;
        }
    });
    return GNN_OK;
}

// Concatenate the sub-graphs and build the sender CSR, the copy list, the edge
// tiles and the per-row positions.
int assemble(const gnn_graph* g, int32_t R, LocalGraphs& LG, gnn_partition* P) {
    P->R = R;
    P->row_offsets.assign(R + 1, 0);
    P->edge_offsets.assign(R + 1, 0);
    for (int r = 0; r < R; ++r) {
        P->row_offsets[r + 1] = P->row_offsets[r] + (int64_t)LG.nodes[r].size();
        P->edge_offsets[r + 1] = P->edge_offsets[r] + (int64_t)LG.lcol[r].size();
    }
    const int64_t NR = P->row_offsets[R], NE = P->edge_offsets[R];
    GNN_REQUIRE(NR < (int64_t)std::numeric_limits<int32_t>::max() &&
                    NE < (int64_t)std::numeric_limits<int32_t>::max(),
                GNN_ESHAPE, "gnn_partition: more than 2^31-1 rows or edges");
    for (int r = 0; r < R; ++r) {
        for (int32_t d : LG.ndeg[r])
            GNN_REQUIRE(d <= 255, GNN_EUNSUPPORTED, "gnn_partition: a node is held by %d rows (at most 255)", d);
        for (int32_t d : LG.ldeg[r])
            GNN_REQUIRE(d <= 255, GNN_EUNSUPPORTED, "gnn_partition: an edge is held by %d sub-graphs (at most 255)", d);
    }
    P->row_gid.resize(NR);
    P->row_ptr.resize(NR + 1);
    P->col.resize(NE);
    P->edge_deg.resize(NE);
    P->node_deg.resize(NR);
    P->row_ptr[0] = 0;
    parallel_for(R, [&](int64_t r) {
        int64_t ro = P->row_offsets[r], eo = P->edge_offsets[r];
        for (size_t i = 0; i < LG.nodes[r].size(); ++i) {
            P->row_gid[ro + i] = LG.nodes[r][i];
            P->node_deg[ro + i] = (uint8_t)LG.ndeg[r][i];
            P->row_ptr[ro + i + 1] = (int32_t)(eo + LG.lptr[r][i + 1]);
        }
        for (size_t t = 0; t < LG.lcol[r].size(); ++t) {
            P->col[eo + t] = (int32_t)(ro + LG.lcol[r][t]);
            P->edge_deg[eo + t] = (uint8_t)LG.ldeg[r][t];
        }
    });
    LG.reset(0);
    int32_t maxdeg = 0;
    for (int64_t i = 0; i < NR; ++i) maxdeg = std::max(maxdeg, P->row_ptr[i + 1] - P->row_ptr[i]);
    P->max_in_degree = maxdeg;

    // ---- sender CSR (counting sort by sender row, edge ids ascending)
    P->t_ptr.assign(NR + 1, 0);
    for (int64_t t = 0; t < NE; ++t) P->t_ptr[P->col[t] + 1]++;
    for (int64_t i = 0; i < NR; ++i) P->t_ptr[i + 1] += P->t_ptr[i];
    P->t_eid.resize(NE);
    {
        std::vector<int32_t> fill(P->t_ptr.begin(), P->t_ptr.end() - 1);
        for (int64_t t = 0; t < NE; ++t) P->t_eid[fill[P->col[t]]++] = (int32_t)t;
    }

    // ---- copy list of shared global ids, copies in increasing row (sub-graph) order
    std::vector<std::pair<int64_t, int32_t>> shared;
    for (int64_t i = 0; i < NR; ++i)
        if (P->node_deg[i] > 1) shared.emplace_back(P->row_gid[i], (int32_t)i);
    std::sort(shared.begin(), shared.end());
    P->halo_ptr.clear();
    P->halo_rows.resize(shared.size());
    P->part_stats.assign((size_t)R * 3, 0);
    std::vector<int32_t> row_part(NR);
    for (int r = 0; r < R; ++r)
        for (int64_t i = P->row_offsets[r]; i < P->row_offsets[r + 1]; ++i) row_part[i] = r;
    std::vector<std::vector<int32_t>> neigh(R);
    for (size_t s = 0; s < shared.size();) {
        size_t e = s;
        while (e < shared.size() && shared[e].first == shared[s].first) ++e;
        GNN_REQUIRE((int64_t)(e - s) == P->node_deg[shared[s].second], GNN_EHALO,
                    "gnn_partition: copy count of gid %lld differs from its degree", (long long)shared[s].first);
        P->halo_ptr.push_back((int32_t)s);
        for (size_t k = s; k < e; ++k) {
            P->halo_rows[k] = shared[k].second;
            int32_t rk = row_part[shared[k].second];
            for (size_t m = s; m < e; ++m) {
                const int32_t rm = row_part[shared[m].second];
                if (rm == rk) continue;      // copies of a split node within one sub-graph
                P->part_stats[rk * 3 + 1] += 1;
                neigh[rk].push_back(rm);
            }
        }
        s = e;
    }
    P->halo_ptr.push_back((int32_t)shared.size());
    for (int r = 0; r < R; ++r) {
        P->part_stats[r * 3 + 0] = P->row_offsets[r + 1] - P->row_offsets[r];
        std::sort(neigh[r].begin(), neigh[r].end());
        P->part_stats[r * 3 + 2] = (int64_t)(std::unique(neigh[r].begin(), neigh[r].end()) - neigh[r].begin());
    }

    // ---- receiver-aligned edge tiles of <= GNN_EDGE_TILE edges, one record each
    GNN_REQUIRE(maxdeg <= GNN_EDGE_TILE, GNN_EHALO, "gnn_partition: in-degree %d after the split exceeds %d",
                maxdeg, GNN_EDGE_TILE);
    build_edge_tiles(P, GNN_EDGE_TILE);
    // ---- positions per row
    P->row_pos.resize(NR * 3);
    for (int64_t i = 0; i < NR; ++i)
        for (int a = 0; a < 3; ++a) P->row_pos[i * 3 + a] = g->pos[P->row_gid[i] * 3 + a];
    return GNN_OK;
}

int partition_core(const gnn_graph* g, int32_t R, const std::vector<int32_t>& part, gnn_partition** out) {
    gnn_partition* P = new (std::nothrow) gnn_partition();
    GNN_REQUIRE(P, GNN_ENOMEM, "gnn_partition: out of host memory");
    int rc;
    try {
        std::vector<int64_t> elem_count(R, 0);
        for (int32_t r : part) elem_count[r]++;
        rc = GNN_OK;
        for (int r = 0; r < R && rc == GNN_OK; ++r)
            if (elem_count[r] == 0) rc = set_error(GNN_EINVAL, "gnn_partition: part %d has no element", r);
        LocalGraphs LG;
        if (rc == GNN_OK)
            rc = g->kind == GNN_GRAPH_BRICK ? local_graphs_brick(g, R, part, LG) : local_graphs_elements(g, R, part, LG);
        if (rc == GNN_OK) rc = split_hubs(LG, R, GNN_EDGE_TILE);
        if (rc == GNN_OK) rc = assemble(g, R, LG, P);
    } catch (const std::bad_alloc&) {
        rc = set_error(GNN_ENOMEM, "gnn_partition: out of host memory");
    }
    if (rc != GNN_OK) {
        delete P;
        return rc;
    }
    *out = P;
    gnn::clear_error();
    return GNN_OK;
}

}  // namespace

extern "C" {

int gnn_partition_halo(const gnn_graph* g, int32_t R, int32_t method, const double* target_weights,
                       gnn_partition** out) {
    GNN_REQUIRE(g && out, GNN_EINVAL, "gnn_partition_halo: NULL argument");
    *out = nullptr;
    const int64_t n_elem = g->n_elem;
    GNN_REQUIRE(R >= 1 && R <= 65535 && R <= n_elem, GNN_EINVAL,
                "gnn_partition_halo: R=%d must be in 1..min(65535, n_elem)", R);
    GNN_REQUIRE(method == GNN_PART_SLAB_Z || method == GNN_PART_RCB, GNN_EINVAL,
                "gnn_partition_halo: unknown method %d", method);
    GNN_REQUIRE(method != GNN_PART_SLAB_Z || g->kind != GNN_GRAPH_BRICK || R <= g->nel[2], GNN_EINVAL,
                "gnn_partition_halo: slab partition needs R <= nel[2]");
    std::vector<double> w(R, 1.0);
    if (target_weights) {
        for (int r = 0; r < R; ++r) {
            GNN_REQUIRE(target_weights[r] > 0.0 && std::isfinite(target_weights[r]), GNN_EINVAL,
                        "gnn_partition_halo: target weight %d not positive", r);
            w[r] = target_weights[r];
        }
    }
    std::vector<int32_t> part;
    try {
        part.assign(n_elem, 0);
        if (method == GNN_PART_SLAB_Z && g->kind == GNN_GRAPH_BRICK) {
            for (int64_t e = 0; e < n_elem; ++e) {
                int64_t ez = e / ((int64_t)g->nel[0] * g->nel[1]);
                int32_t r = 0;
                while (r + 1 < R && ez >= ((int64_t)(r + 1) * g->nel[2]) / R) ++r;
                part[e] = r;
            }
        } else if (method == GNN_PART_SLAB_Z) {
            std::vector<int64_t> order(n_elem);
            for (int64_t e = 0; e < n_elem; ++e) order[e] = e;
            std::sort(order.begin(), order.end(), [&](int64_t u, int64_t v) {
                double cu = g->centre[u * 3 + 2], cv = g->centre[v * 3 + 2];
                if (cu != cv) return cu < cv;
                return u < v;
            });
            int32_t r = 0;
            for (int64_t s = 0; s < n_elem; ++s) {
                while (r + 1 < R && s >= ((int64_t)(r + 1) * n_elem) / R) ++r;
                part[order[s]] = r;
            }
        } else {
            std::vector<double> centre;
            if (g->kind == GNN_GRAPH_BRICK) {
                centre.resize(n_elem * 3);
                double h[3];
                for (int a = 0; a < 3; ++a) h[a] = g->extent[a] / g->nel[a];
                for (int64_t e = 0; e < n_elem; ++e) {
                    int64_t c[3] = {e % g->nel[0], (e / g->nel[0]) % g->nel[1], e / ((int64_t)g->nel[0] * g->nel[1])};
                    for (int a = 0; a < 3; ++a) centre[e * 3 + a] = (c[a] + 0.5) * h[a];
                }
            }
            std::vector<int64_t> elems(n_elem);
            for (int64_t e = 0; e < n_elem; ++e) elems[e] = e;
            rcb_split(g->kind == GNN_GRAPH_BRICK ? centre : g->centre, elems, 0, n_elem, 0, R, w, part);
        }
    } catch (const std::bad_alloc&) {
        return set_error(GNN_ENOMEM, "gnn_partition_halo: out of host memory");
    }
    return partition_core(g, R, part, out);
}

int gnn_partition_elements(const gnn_graph* g, int32_t R, const int32_t* elem_part, gnn_partition** out) {
    GNN_REQUIRE(g && elem_part && out, GNN_EINVAL, "gnn_partition_elements: NULL argument");
    *out = nullptr;
    GNN_REQUIRE(R >= 1 && R <= 65535 && R <= g->n_elem, GNN_EINVAL,
                "gnn_partition_elements: R=%d must be in 1..min(65535, n_elem)", R);
    std::vector<int32_t> part;
    try {
        part.assign(elem_part, elem_part + g->n_elem);
    } catch (const std::bad_alloc&) {
        return set_error(GNN_ENOMEM, "gnn_partition_elements: out of host memory");
    }
    for (int64_t e = 0; e < g->n_elem; ++e)
        GNN_REQUIRE(part[e] >= 0 && part[e] < R, GNN_EINVAL, "gnn_partition_elements: element %lld part %d out of range",
                    (long long)e, part[e]);
    return partition_core(g, R, part, out);
}

void gnn_partition_destroy(gnn_partition* p) { delete p; }

int gnn_partition_get_info(const gnn_partition* P, gnn_partition_info* info) {
    GNN_REQUIRE(P && info, GNN_EINVAL, "gnn_partition_get_info: NULL argument");
    info->n_parts = P->R;
    info->max_in_degree = P->max_in_degree;
    info->n_rows = (int64_t)P->row_gid.size();
    info->n_edges = (int64_t)P->col.size();
    info->n_shared = (int64_t)P->halo_ptr.size() - 1;
    info->n_copies = (int64_t)P->halo_rows.size();
    info->n_edge_tiles = (int64_t)P->edge_tiles.size() - 1;
    info->n_node_tiles = (info->n_rows + GNN_NODE_TILE - 1) / GNN_NODE_TILE;
    info->tile_edges = P->tile_edges;
    info->reserved = 0;
    return GNN_OK;
}

int gnn_partition_set_tile_edges(gnn_partition* P, int32_t tile_edges) {
    GNN_REQUIRE(P, GNN_EINVAL, "gnn_partition_set_tile_edges: NULL partition");
    GNN_REQUIRE(tile_edges >= std::max(P->max_in_degree, 1) && tile_edges <= GNN_EDGE_TILE, GNN_EINVAL,
                "gnn_partition_set_tile_edges: tile_edges %d outside [%d, %d]", tile_edges,
                std::max(P->max_in_degree, 1), GNN_EDGE_TILE);
    try {
        build_edge_tiles(P, tile_edges);
    } catch (const std::bad_alloc&) {
        return set_error(GNN_ENOMEM, "gnn_partition_set_tile_edges: out of host memory");
    }
    return GNN_OK;
}

int gnn_partition_copy(const gnn_partition* P, int32_t what, void* dst, size_t bytes) {
    GNN_REQUIRE(P && (dst || bytes == 0), GNN_EINVAL, "gnn_partition_copy: NULL argument");
    const void* src = nullptr;
    size_t n = 0;
    std::vector<float> tmp;
    switch (what) {
        case GNN_P_ROW_OFFSETS: src = P->row_offsets.data(); n = P->row_offsets.size() * 8; break;
        case GNN_P_EDGE_OFFSETS: src = P->edge_offsets.data(); n = P->edge_offsets.size() * 8; break;
        case GNN_P_ROW_GID: src = P->row_gid.data(); n = P->row_gid.size() * 8; break;
        case GNN_P_ROW_PTR: src = P->row_ptr.data(); n = P->row_ptr.size() * 4; break;
        case GNN_P_COL: src = P->col.data(); n = P->col.size() * 4; break;
        case GNN_P_EDGE_DEG: src = P->edge_deg.data(); n = P->edge_deg.size(); break;
        case GNN_P_NODE_DEG: src = P->node_deg.data(); n = P->node_deg.size(); break;
        case GNN_P_EDGE_W:
            tmp.resize(P->edge_deg.size());
            for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = 1.0f / (float)P->edge_deg[i];
            src = tmp.data(); n = tmp.size() * 4; break;
        case GNN_P_NODE_W:
            tmp.resize(P->node_deg.size());
            for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = 1.0f / (float)P->node_deg[i];
            src = tmp.data(); n = tmp.size() * 4; break;
        case GNN_P_T_PTR: src = P->t_ptr.data(); n = P->t_ptr.size() * 4; break;
        case GNN_P_T_EID: src = P->t_eid.data(); n = P->t_eid.size() * 4; break;
        case GNN_P_HALO_PTR: src = P->halo_ptr.data(); n = P->halo_ptr.size() * 4; break;
        case GNN_P_HALO_ROWS: src = P->halo_rows.data(); n = P->halo_rows.size() * 4; break;
        case GNN_P_EDGE_TILES: src = P->edge_tiles.data(); n = P->edge_tiles.size() * 4; break;
        case GNN_P_ROW_POS: src = P->row_pos.data(); n = P->row_pos.size() * 8; break;
        case GNN_P_PART_STATS: src = P->part_stats.data(); n = P->part_stats.size() * 8; break;
        case GNN_P_TILE_META: src = P->tile_meta.data(); n = P->tile_meta.size(); break;
        case GNN_P_EDGE_ATTR: {
            const int64_t NR = (int64_t)P->row_gid.size();
            tmp.resize(P->col.size() * 4);
            for (int64_t i = 0; i < NR; ++i)
                for (int32_t t = P->row_ptr[i]; t < P->row_ptr[i + 1]; ++t) {
                    const double* pr = &P->row_pos[i * 3];
                    const double* ps = &P->row_pos[(int64_t)P->col[t] * 3];
                    double dx = ps[0] - pr[0], dy = ps[1] - pr[1], dz = ps[2] - pr[2];
                    tmp[(size_t)t * 4 + 0] = (float)dx;
                    tmp[(size_t)t * 4 + 1] = (float)dy;
                    tmp[(size_t)t * 4 + 2] = (float)dz;
                    tmp[(size_t)t * 4 + 3] = (float)std::sqrt(dx * dx + dy * dy + dz * dz);
                }
            src = tmp.data(); n = tmp.size() * 4; break;
        }
        default: return set_error(GNN_EINVAL, "gnn_partition_copy: unknown array %d", what);
    }
    GNN_REQUIRE(bytes == n, GNN_ESHAPE, "gnn_partition_copy: array %d has %zu bytes, buffer %zu", what, n, bytes);
    if (n) std::memcpy(dst, src, n);
    return GNN_OK;
}

}  // extern "C"
