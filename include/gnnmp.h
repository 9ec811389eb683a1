/*
 * gnnmp.h -- C ABI of libgnnmp: the consistent neural message-passing (NMP)
 * layer of arXiv 2410.01657 ("Scalable and Consistent Graph Neural Networks
 * for Distributed Mesh-based Data-driven Modeling") on one GB300 (sm_103a).
 *
 * Conventions for every entry point
 *  - Return 0 (GNN_OK) on success or a negative GNN_E* code; the thread-local
 *    message of the last failure is gnn_last_error(). No C++ exception crosses
 *    this boundary.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA global
 *    memory of the current device. The caller allocates and owns every device
 *    buffer passed in (PyTorch does it in the Python binding); the library
 *    allocates device memory nowhere in the compute calls.
 *  - Compute calls are asynchronous on the CUDA stream passed as `stream`
 *    (a cudaStream_t cast to void*, NULL = legacy default stream). Argument
 *    errors are reported synchronously; a kernel-side failure (a bounded wait
 *    that ran out, a bounds check) is latched in a device error word and
 *    reported by the next gnn_check().
 *  - Matrices are row-major. Node rows [n_rows x H] and edge rows
 *    [n_edges x H] follow the row and edge order of the gnn_partition they
 *    were built for (partitions concatenated, receiver-sorted edges).
 */
#ifndef GNNMP_H
#define GNNMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define GNN_OK            0
#define GNN_EINVAL       -1   /* bad argument (NULL pointer, out-of-range value)        */
#define GNN_ESHAPE       -2   /* inconsistent sizes or a size the kernels cannot take   */
#define GNN_EDTYPE       -3   /* unsupported precision / dtype combination              */
#define GNN_ECUDA        -4   /* a CUDA runtime or driver call failed                   */
#define GNN_EHALO        -5   /* inconsistent partition / halo bookkeeping              */
#define GNN_ETIMEOUT     -6   /* a bounded device-side wait ran out (see gnn_check)     */
#define GNN_ENOMEM       -7   /* host allocation failed or workspace too small          */
#define GNN_EUNSUPPORTED -8   /* valid input the implementation does not cover          */

/* Message of the last failed call on this thread ("" if none). */
const char* gnn_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int gnn_version(void);
/* Synchronise `stream`, then read and clear the device error words (one per
 * source file of kernels that wait). Returns GNN_OK, GNN_ETIMEOUT (a device
 * wait gave up; gnn_last_error() names the source files whose kernels timed
 * out) or GNN_ECUDA. */
int gnn_check(void* stream);

/* ====================================================== graph generation (host)
 * Sec. II-A, Fig. 2: nodes at the GLL quadrature points of hexahedral elements
 * of polynomial order p, undirected edges between neighbouring quadrature
 * points of an element (6-neighbour stencil, both directions), coincident
 * nodes of neighbouring elements merged by global id.
 */
typedef struct gnn_mesh_desc {
    int32_t nel[3];          /* elements per axis (>= 1)                                  */
    int32_t p;               /* polynomial order (1..15)                                  */
    double extent[3];        /* brick [0,extent[a]]; element size extent[a]/nel[a]        */
    int32_t periodic[3];     /* nonzero: axis wraps (needs nel*p >= 3)                    */
    double jitter_frac;      /* node displacement as a fraction of the local GLL spacing  */
    const double* jitter;    /* host [n_nodes x 3] values in [-1,1], or NULL (no jitter)  */
} gnn_mesh_desc;

typedef struct gnn_graph gnn_graph;   /* opaque, library-owned host object */

#define GNN_GRAPH_BRICK    0   /* built by gnn_graph_build                                  */
#define GNN_GRAPH_ELEMENTS 1   /* built by gnn_graph_build_elements                         */

typedef struct gnn_graph_info {
    int64_t n_nodes;         /* brick: lattice points, prod(L)                            */
    int64_t n_edges;         /* directed edges of the R=1 graph                           */
    int64_t n_elem;
    int32_t L[3];            /* brick: lattice points per axis, nel*p (+1 if not periodic); 0 otherwise */
    int32_t p;               /* brick: polynomial order; 0 otherwise                      */
    int64_t n_elem_nodes;    /* entries of the element node lists (brick: n_elem*(p+1)^3) */
    int32_t kind;            /* GNN_GRAPH_*                                               */
    int32_t max_degree;      /* largest in-degree of the R=1 graph                        */
} gnn_graph_info;

/* Build the R=1 GLL-brick graph. Global id of lattice point (ix,iy,iz) is
 * ix + L0*(iy + L1*iz); the CSR is receiver-sorted, senders ascending.
 * Node (ix,..) moves by jitter[g*3+a]*jitter_frac*(smallest adjacent GLL
 * spacing on axis a), except the normal coordinate on non-periodic faces.
 * *out is freed with gnn_graph_destroy. Errors: GNN_EINVAL, GNN_ENOMEM. */
int gnn_graph_build(const gnn_mesh_desc* desc, gnn_graph** out);

/* General element meshes. Sec. II-A notes that the graph construction and its
 * distribution apply to any mesh made of finite elements; here elements of any
 * type and size may be mixed. Element e holds the global node ids
 * elem_nodes[elem_ptr[e] .. elem_ptr[e+1]) and the undirected edges joining
 * its local nodes u and v for every pair (u, v) = (edge_pairs[2k],
 * edge_pairs[2k+1]), k in [edge_ptr[e], edge_ptr[e+1]) -- a hex of order p
 * lists its (p+1)^3 GLL nodes and stencil pairs, a tetrahedron its 4 vertices
 * and 6 edges, a polyhedral cell with a centre node the spokes from it. The
 * R=1 graph is the union of the element edges in both directions (receiver-
 * sorted, senders ascending; a node's in-degree is not bounded). An element's
 * centre, which GNN_PART_RCB and GNN_PART_SLAB_Z split, is the mean position
 * of its nodes. The arrays are read during the call only.
 * Errors: GNN_EINVAL (NULL arrays, offsets not starting at 0 or descending, a
 * node id or local index out of range, a pair joining a node to itself, a node
 * in no element or on no edge -- every row of a partition then receives at
 * least one edge, as the edge kernels expect), GNN_ESHAPE (more than 2^31-1
 * nodes), GNN_ENOMEM. */
typedef struct gnn_elem_mesh_desc {
    int64_t n_nodes;
    const double* pos;          /* host [n_nodes x 3] node positions                         */
    int64_t n_elem;
    const int64_t* elem_ptr;    /* host [n_elem+1] offsets into elem_nodes                   */
    const int64_t* elem_nodes;  /* host [elem_ptr[n_elem]] global node ids, 0 <= id < n_nodes */
    const int64_t* edge_ptr;    /* host [n_elem+1] offsets into edge_pairs, in pairs         */
    const int32_t* edge_pairs;  /* host [2 x edge_ptr[n_elem]] element-local node indices    */
} gnn_elem_mesh_desc;
int gnn_graph_build_elements(const gnn_elem_mesh_desc* desc, gnn_graph** out);

void gnn_graph_destroy(gnn_graph* g);
int gnn_graph_get_info(const gnn_graph* g, gnn_graph_info* info);
/* Copy-out accessors into caller-owned host buffers of the stated length. */
int gnn_graph_copy_pos(const gnn_graph* g, double* pos /* [n_nodes*3] */);
int gnn_graph_copy_csr(const gnn_graph* g, int64_t* row_ptr /* [n_nodes+1] */,
                       int64_t* col /* [n_edges] */);
/* Element node lists, concatenated ([n_elem_nodes]; a brick element's (p+1)^3
 * nodes in local order i + (p+1)*(j + (p+1)*k)), and their offsets. */
int gnn_graph_copy_elements(const gnn_graph* g, int64_t* elem_nodes /* [n_elem_nodes] */);
int gnn_graph_copy_element_ptr(const gnn_graph* g, int64_t* elem_ptr /* [n_elem+1] */);

/* ================================================ partitioning + halo (host)
 * Sec. II-A, Figs. 3-4: elements are split over R sub-graphs; each keeps the
 * nodes and stencil edges of its own elements with local coincident nodes
 * collapsed (the "reduced" graph). d_ij (Eq. 5b) counts the sub-graphs that
 * hold directed edge (i,j); d_i (Eq. 8b) the sub-graphs that hold node i.
 * On one GPU all sub-graphs are resident as one concatenated row space, so the
 * halo rows of Fig. 4 become a copy list: for every global id held by >= 2
 * sub-graphs, the rows holding it in increasing sub-graph order.
 */
#define GNN_PART_SLAB_Z 0    /* R contiguous z-layers of elements (element meshes: R
                                 runs of the elements sorted by (centre z, id), run r
                                 holding sorted positions [floor(r*n/R), floor((r+1)*n/R))) */
#define GNN_PART_RCB    1    /* recursive coordinate bisection of element centres        */

typedef struct gnn_partition gnn_partition;   /* opaque, library-owned host object */

typedef struct gnn_partition_info {
    int32_t n_parts;         /* R                                                          */
    int32_t max_in_degree;   /* largest receiver in-degree over all rows (<= GNN_EDGE_TILE) */
    int64_t n_rows;          /* sum of local rows over sub-graphs                          */
    int64_t n_edges;         /* sum of local directed edges                                */
    int64_t n_shared;        /* global ids held by >= 2 sub-graphs                        */
    int64_t n_copies;        /* rows holding those ids (length of the copy list)          */
    int64_t n_edge_tiles;    /* receiver-aligned tiles of <= tile_edges edges              */
    int64_t n_node_tiles;    /* tiles of GNN_NODE_TILE consecutive rows                    */
    int32_t tile_edges;      /* edge cap of the edge tiles (GNN_EDGE_TILE unless re-tiled) */
    int32_t reserved;
} gnn_partition_info;

#define GNN_EDGE_TILE 128
#define GNN_NODE_TILE 128

/* Partition g into R sub-graphs. method is GNN_PART_*; target_weights (host,
 * R positive doubles, NULL = equal) sets the RCB share of each part. RCB
 * splits a set of parts [r0, r0+n) into its first floor(n/2) parts and the
 * rest along the axis of largest element-centre extent (lowest axis on ties),
 * after a stable sort by (centre, element id), giving the left side
 * floor(count*W_left/W + 0.5) elements (at least one per part).
 * Brick elements have their lattice centres; element-mesh elements the mean
 * of their node positions.
 * Errors: GNN_EINVAL (R out of range, bad weights), GNN_ESHAPE (more than
 * 2^31-1 rows or edges), GNN_EUNSUPPORTED (a node or edge held by more than
 * 255 rows or sub-graphs), GNN_ENOMEM. */
int gnn_partition_halo(const gnn_graph* g, int32_t R, int32_t method,
                       const double* target_weights, gnn_partition** out);
/* Partition g with a caller-given element -> sub-graph map (host [n_elem]
 * values in [0, R), every sub-graph non-empty), e.g. a solver's own domain
 * decomposition. Everything else as gnn_partition_halo.
 * Errors: GNN_EINVAL (R out of range, a value out of range, an empty part),
 * GNN_ESHAPE, GNN_EUNSUPPORTED, GNN_ENOMEM. */
int gnn_partition_elements(const gnn_graph* g, int32_t R, const int32_t* elem_part,
                           gnn_partition** out);

/* Nodes of high in-degree. The edge kernels take tiles of whole receivers
 * (GNN_EDGE_TILE edges at most), so a node whose in-degree within one
 * sub-graph exceeds GNN_EDGE_TILE is held there by k = ceil(degree /
 * GNN_EDGE_TILE) consecutive rows (copies), copy c receiving the c-th of k
 * near-equal consecutive runs of its in-edges (senders ascending) and sending
 * to the nodes of that run. The copies enter the copy list like the copies in
 * other sub-graphs, so Eq. 5c-5d sums their partial aggregates (the carry of
 * the split receiver) and every copy continues with the same a*; d_i (Eq. 8b)
 * counts all rows holding node i. Rows within a sub-graph stay ordered by
 * global id. GNN_EUNSUPPORTED when a node would need more than 255 rows in
 * total (d_i and d_ij are 8-bit). */
void gnn_partition_destroy(gnn_partition* p);
int gnn_partition_get_info(const gnn_partition* p, gnn_partition_info* info);

/* Rebuild the edge tiles of p (GNN_P_EDGE_TILES, GNN_P_TILE_META) with at
 * most `tile_edges` edges and GNN_EDGE_TILE rows per tile; rows never straddle
 * two tiles. Smaller tiles trade per-tile overhead for more parallel work on
 * small graphs (a launch-shape choice: results do not depend on it).
 * Device copies made earlier keep the old tiles; upload again afterwards.
 * Errors: GNN_EINVAL unless max_in_degree <= tile_edges <= GNN_EDGE_TILE. */
int gnn_partition_set_tile_edges(gnn_partition* p, int32_t tile_edges);

/* Arrays of a partition, copied into a caller-owned host buffer of exactly
 * `bytes` bytes (GNN_ESHAPE otherwise). Row r of sub-graph s is global row
 * row_offsets[s] + r; local rows are ordered by global id (the copies of a
 * split high in-degree node are consecutive). */
#define GNN_P_ROW_OFFSETS  0   /* int64 [R+1]                                               */
#define GNN_P_EDGE_OFFSETS 1   /* int64 [R+1]                                               */
#define GNN_P_ROW_GID      2   /* int64 [n_rows] global id of each row                      */
#define GNN_P_ROW_PTR      3   /* int32 [n_rows+1] receiver CSR                             */
#define GNN_P_COL          4   /* int32 [n_edges] sender row (same sub-graph), ascending gid */
#define GNN_P_EDGE_DEG     5   /* uint8 [n_edges] d_ij                                      */
#define GNN_P_EDGE_W       6   /* float [n_edges] 1/d_ij                                    */
#define GNN_P_NODE_DEG     7   /* uint8 [n_rows] d_i                                        */
#define GNN_P_NODE_W       8   /* float [n_rows] 1/d_i                                      */
#define GNN_P_T_PTR        9   /* int32 [n_rows+1] sender CSR                               */
#define GNN_P_T_EID       10   /* int32 [n_edges] edge ids by sender, ascending             */
#define GNN_P_HALO_PTR    11   /* int32 [n_shared+1]                                        */
#define GNN_P_HALO_ROWS   12   /* int32 [n_copies] rows of each shared id, by sub-graph     */
#define GNN_P_EDGE_TILES  13   /* int32 [n_edge_tiles+1] first receiver row of each tile    */
#define GNN_P_EDGE_ATTR   14   /* float [n_edges*4] [dx,dy,dz,|d|], d = pos(send)-pos(recv) */
#define GNN_P_ROW_POS     15   /* double [n_rows*3]                                         */
#define GNN_P_PART_STATS  16   /* int64 [R*3] per sub-graph: local rows, halo rows, neighbours */
#define GNN_P_TILE_META   17   /* uint8 [n_edge_tiles * GNN_TILE_META_BYTES] per-tile records   */

/* Per-edge-tile record (GNN_P_TILE_META), one 2 KiB block per tile so a kernel
 * can fetch a tile's bookkeeping with one bulk copy: bytes 0..15 int32
 * {first row r0, end row r1, first edge e0, edge count ne}; 16..543 int32
 * rp[132] = row_ptr[r0+i] - e0 for i <= r1-r0; 544..799 int16 seg[128] =
 * local receiver row of each edge; 800..1311 int32 col[128] = sender row;
 * 1312..1823 float w[128] = 1/d_ij; the rest zero. */
#define GNN_TILE_META_BYTES 2048
int gnn_partition_copy(const gnn_partition* p, int32_t what, void* dst, size_t bytes);

/* ====================================================== device-side graph
 * The arrays above after upload to device memory by the caller. Pointers are
 * device pointers, borrowed for the duration of each call.
 */
typedef struct gnn_graph_dev {
    int64_t n_rows;
    int64_t n_edges;
    const int32_t* row_ptr;     /* [n_rows+1]   */
    const int32_t* col;         /* [n_edges]    */
    const float*   edge_w;      /* [n_edges]    1/d_ij                                      */
    const int32_t* t_ptr;       /* [n_rows+1]   */
    const int32_t* t_eid;       /* [n_edges]    */
    const float*   node_w;      /* [n_rows]     1/d_i (consistent loss)                     */
    int64_t n_shared;
    const int32_t* halo_ptr;    /* [n_shared+1] */
    const int32_t* halo_rows;   /* [n_copies]   */
    int64_t n_edge_tiles;
    const int32_t* edge_tiles;  /* [n_edge_tiles+1] */
    int32_t max_in_degree;      /* host copy of gnn_partition_info.max_in_degree            */
    const void*    tile_meta;   /* [n_edge_tiles * GNN_TILE_META_BYTES], 16-byte aligned    */
} gnn_graph_dev;

/* ====================================================== parameters
 * One MLP block (Sec. III, Table 1): n_lin = n_hidden + 2 Linear layers
 * dims[0] -> dims[1] -> ... -> dims[n_lin], ELU (alpha 1) after all but the
 * last, then an affine LayerNorm over dims[n_lin] when gamma != NULL. W[k] is
 * [dims[k+1] x dims[k]] row-major (out x in), FP32 device memory. The same
 * struct carries gradients (dW, db, dgamma, dbeta), which calls accumulate into.
 */
#define GNN_MAX_LIN 8
typedef struct gnn_mlp {
    int32_t n_lin;
    int32_t dims[GNN_MAX_LIN + 1];
    float* W[GNN_MAX_LIN];
    float* b[GNN_MAX_LIN];
    float* gamma;               /* NULL: no LayerNorm */
    float* beta;
} gnn_mlp;

/* One consistent NMP layer: edge MLP on [x_i, x_j, e_ij] (3H -> H) and node
 * MLP on [a*_i, x_i] (2H -> H), both with LayerNorm (Eq. 5a, 5e). */
typedef struct gnn_mp_params {
    gnn_mlp edge;
    gnn_mlp node;
} gnn_mp_params;

#define GNN_PREC_FP32 0   /* plain FP32 SIMT kernels, FP32 edge state                       */
#define GNN_PREC_BF16 1   /* fused tcgen05 kernels: BF16 GEMM operands, FP32 accumulation,
                             FP32 sums/LayerNorm statistics, BF16 edge state and edge grads */
#define GNN_HALO_SYNC 0   /* consistent layer (Eq. 5c-5d applied)                           */
#define GNN_HALO_NONE 1   /* the paper's "None" mode: Eq. 5c-5d skipped (inconsistent)     */
#define GNN_FLAG_NO_EDGE_OUT 1  /* forward: do not write e_out (last layer in inference)  */
#define GNN_FLAG_ADJ_ONE_LINEAR 2  /* backward, BF16 at H = 128: one Linear per adjoint pass
                                     instead of two, and the first Linear's edge part in a
                                     pass of its own (same results, bit for bit; for testing) */

/* Launch choices of the fused BF16 edge forward. Every choice computes the
 * same arithmetic; FP32 results agree to rounding (instruction pairing and
 * contraction differ), so a value rounded to BF16 afterwards (edge state, MMA
 * operands) can differ in its last bit. 0 = library default. */
#define GNN_EDGE_FWD_AUTO 0   /* RT for H <= 64, TM for H = 128 (ONE beyond 2 MLP hidden layers) */
#define GNN_EDGE_FWD_RT   1   /* record-tiled consumer groups, P|Q rows prefetched (H <= 64)   */
#define GNN_EDGE_FWD_WS   2   /* producer warp + two consumer groups (H <= 64)                 */
#define GNN_EDGE_FWD_ONE  3   /* one tile at a time per CTA, CTAs per SM by occupancy          */
#define GNN_EDGE_FWD_TM   4   /* two tile groups per SM, hidden activations kept in tensor
                                 memory as the next Linear's operand (H = 128, <= 4 Linears) */

typedef struct gnn_mp_config {
    int32_t hidden;          /* H: 16, 32, 64 or 128 (BF16); 1..256 (FP32)                 */
    int32_t precision;       /* GNN_PREC_*                                                  */
    int32_t halo_mode;       /* GNN_HALO_*                                                  */
    int32_t flags;           /* GNN_FLAG_*                                                  */
    float ln_eps;            /* LayerNorm epsilon (the paper's PyTorch default 1e-5)       */
    int32_t edge_fwd_kernel; /* GNN_EDGE_FWD_* (BF16 only; ignored for FP32)               */
    int32_t ctas_per_sm;     /* cap on resident CTAs per SM of the BF16 edge forward;
                                0 = as many as shared memory, registers and TMEM allow   */
} gnn_mp_config;

/* ====================================================== consistent NMP layer
 * Workspace bytes needed by gnn_mp_forward / gnn_mp_backward for this graph,
 * configuration and parameter shapes. */
int gnn_mp_workspace_size(const gnn_graph_dev* G, const gnn_mp_config* cfg,
                          const gnn_mp_params* W, size_t* fwd_bytes, size_t* bwd_bytes);

/* Forward of one consistent NMP layer, Eq. 5a-5e:
 *   e'_ij = e_ij + LN(MLP_E([x_i, x_j, e_ij]))   (i receiver, j sender)     Eq. 5a
 *   a_i   = sum_j e'_ij / d_ij                    (FP32, fixed order)        Eq. 5b
 *   a*_i  = sum over the copies of node i of a    (halo swap + sync)         Eq. 5c-5d
 *   x'_i  = x_i + LN(MLP_N([a*_i, x_i]))                                     Eq. 5e
 * x_in/x_out: device FP32 [n_rows x H]. e_in/e_out: device [n_edges x H],
 * FP32 for GNN_PREC_FP32, BF16 for GNN_PREC_BF16. a_star_out: device FP32
 * [n_rows x H] or NULL (saved for the backward, which otherwise recomputes it).
 * e_out may be NULL with GNN_FLAG_NO_EDGE_OUT. x_out must not alias x_in.
 * ws: device workspace of ws_bytes >= the forward size. */
int gnn_mp_forward(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                   const float* x_in, const void* e_in, float* x_out, void* e_out,
                   float* a_star_out, void* ws, size_t ws_bytes, void* stream);

/* Backward (adjoint) of gnn_mp_forward with per-layer recomputation of the
 * MLP activations (Eq. 3). Given dL/dx_out and dL/de_out (NULL = zero),
 * writes dL/dx_in (FP32) and dL/de_in (edge dtype) and ACCUMULATES (+=) the
 * parameter gradients into dW (same shapes as W, FP32) in a fixed order.
 * a_star: the forward's a_star_out, or NULL to recompute it. The halo adjoint
 * is the same copy-sum as the forward (the map a -> a* is symmetric).
 * BF16 at H = 128: the MLP adjoints run one Linear at a time over tiles of
 * 128 rows with the recomputed activations in workspace scratch, in chunks
 * of tiles; gnn_mp_workspace_size reports the size for the largest chunk,
 * and a smaller ws_bytes (at least the size for a one-tile chunk) gives more,
 * smaller chunks with the same results. GNN_ENOMEM below that. */
int gnn_mp_backward(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                    const float* x_in, const void* e_in, const float* a_star,
                    const float* dx_out, const void* de_out, float* dx_in, void* de_in,
                    const gnn_mp_params* dW, void* ws, size_t ws_bytes, void* stream);

/* Training with saved activations. The backward above recomputes each MLP
 * chain, which makes its per-tile work a serial run of 2L tensor-core steps;
 * keeping the activations instead -- as the paper's autograd training does --
 * leaves one recomputed Linear per MLP. gnn_mp_forward_act is gnn_mp_forward
 * that also writes the hidden activations h_0 .. h_{L-2} (the ELU outputs,
 * rounded to the BF16 operands of Linears 2..L) of every edge and every node
 * row to act; gnn_mp_backward_act, given that act, reads them by TMA,
 * recomputes only the last Linear of each MLP and needs no P|Q rows. Same
 * results as gnn_mp_forward with GNN_EDGE_FWD_RT (the edge forward it always
 * uses) and gnn_mp_backward. act: device BF16, 16-byte aligned, of
 * gnn_mp_act_size bytes, caller-owned and unchanged from the forward to the
 * backward, in whole 128-row tiles (each tile's rows are stored with one
 * TMA store): edge block k (k < L_e - 1, L_e = W->edge.n_lin) holds row
 * k * T + t * 128 + i for edge row i of edge tile t (T = n_edge_tiles * 128;
 * a tile's rows past its edge count are padding), then node block k
 * (k < L_n - 1) rows k * R + r with R = ceil(n_rows / 128) * 128, then the
 * node MLP's BF16 input rows [a*, x] (R rows, 2H wide). The size
 * depends on the tiling: after gnn_partition_set_tile_edges ask again.
 * gnn_mp_act_size reports 0 where the backward recomputes instead (the FP32
 * path, BF16 at H = 128, whose adjoint is layered, tilings with T above
 * 1.25 n_edges -- edge caps below 128, whose tiles would hold mostly padding
 * -- and graphs with (L_e - 1) * T or (L_n - 1) * R >= 2^31);
 * there act may be NULL and the two calls are
 * gnn_mp_forward / gnn_mp_backward. Errors: those of gnn_mp_forward /
 * gnn_mp_backward; GNN_EINVAL for a NULL or misaligned act that is needed. */
int gnn_mp_act_size(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                    size_t* bytes);
int gnn_mp_forward_act(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                       const float* x_in, const void* e_in, float* x_out, void* e_out,
                       float* a_star_out, void* act, void* ws, size_t ws_bytes, void* stream);
int gnn_mp_backward_act(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                        const float* x_in, const void* e_in, const float* a_star, const void* act,
                        const float* dx_out, const void* de_out, float* dx_in, void* de_in,
                        const gnn_mp_params* dW, void* ws, size_t ws_bytes, void* stream);

/* One timed launch choice of gnn_mp_autotune. */
typedef struct gnn_tune_entry {
    int32_t edge_fwd_kernel;   /* GNN_EDGE_FWD_*                                          */
    int32_t ctas_per_sm;       /* 0 = occupancy limit                                     */
    float ms;                  /* mean device time of one gnn_mp_forward call             */
} gnn_tune_entry;

/* Autotuner of the BF16 layer forward on one graph: times gnn_mp_forward
 * (same arguments as there) for every launch choice of the edge forward that
 * is valid for cfg->hidden, `reps` calls each after one untimed call, with
 * CUDA events on `stream`; writes the fastest choice into cfg->edge_fwd_kernel
 * and cfg->ctas_per_sm and, if out != NULL, up to max_out timings into out
 * (*n_out = number written). Tile shapes are chosen one level up, by timing
 * this call on graphs re-tiled with gnn_partition_set_tile_edges.
 * Synchronises `stream` (not capturable: tune before capturing a graph) and
 * overwrites x_out, e_out and a_star_out. Errors: those of gnn_mp_forward;
 * GNN_EDTYPE for GNN_PREC_FP32, which has no launch choices. */
int gnn_mp_autotune(const gnn_graph_dev* G, gnn_mp_config* cfg, const gnn_mp_params* W,
                    const float* x_in, const void* e_in, float* x_out, void* e_out, float* a_star_out,
                    void* ws, size_t ws_bytes, int32_t reps, gnn_tune_entry* out, int32_t max_out,
                    int32_t* n_out, void* stream);

/* gnn_mp_forward for callers that cannot allocate device memory when they run
 * the layer: code executing while a CUDA stream is being captured without a
 * graph memory pool, or a host framework that owns the device allocator and
 * passes the library only the tensors it computes on. The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Same arguments and results as gnn_mp_forward with GNN_PREC_BF16, minus the
 * workspace: the scratch (P|Q rows, plus the aggregate when a_star_out is
 * NULL) lives in a fixed 64 MiB area compiled into the library, which every
 * GPU that loads the library keeps until the process exits. The area fits
 * about n_rows * 4H bytes of scratch (n_rows * 8H when a_star_out is NULL);
 * larger graphs get GNN_ESHAPE with the required size in gnn_last_error(),
 * before any work is queued. GNN_EDTYPE for GNN_PREC_FP32.
 * Every call outside stream capture looks up the area's device address on
 * the current device; a call made while `stream` is being captured uses the
 * address found by that device's last call outside capture, so make a first
 * call on each device before any capture (GNN_EINVAL otherwise). No call
 * allocates or frees device memory. All calls share the one area and
 * every byte of scratch is written before it is read, so nothing carries over
 * between calls, but calls whose executions overlap on the GPU (two streams,
 * or two host threads) race on it: serialise them. */
int gnn_mp_forward_static(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                          const float* x_in, const void* e_in, float* x_out, void* e_out, float* a_star_out,
                          void* stream);

/* Eq. 5c-5d on one GPU: for every global id held by >= 2 rows, replace each
 * copy by the sum of all copies (summed in increasing sub-graph order, so all
 * copies end bitwise equal). rows: device FP32 [n_rows x width], in place.
 * The map is symmetric, so it is also its own adjoint. */
int gnn_halo_exchange(const gnn_graph_dev* G, float* rows, int32_t width, void* stream);

/* ====================================================== encoder / decoder / loss
 * Row-wise MLP block (node/edge encoders, node decoder; Sec. III): Y = MLP(X)
 * over n_rows rows. X: device FP32 [n_rows x dims[0]]; Y: device
 * [n_rows x dims[n_lin]], FP32 (y_bf16 = 0) or BF16 (y_bf16 = 1).
 * These FP32 calls run over blocks of at most 2^22 rows; the workspace holds
 * one block's activations, so it stays bounded for any n_rows. */
int gnn_mlp_workspace_size(const gnn_mlp* P, int64_t n_rows, size_t* fwd_bytes, size_t* bwd_bytes);
int gnn_mlp_forward(const gnn_mlp* P, int64_t n_rows, const float* X, void* Y, int32_t y_bf16,
                    float ln_eps, void* ws, size_t ws_bytes, void* stream);
/* dY: device [n_rows x dims[n_lin]] FP32 (dy_bf16 = 0) or BF16 (dy_bf16 = 1).
 * dX: device FP32 [n_rows x dims[0]] or NULL. dP accumulates (+=). */
int gnn_mlp_backward(const gnn_mlp* P, int64_t n_rows, const float* X, const void* dY,
                     int32_t dy_bf16, float* dX, const gnn_mlp* dP, float ln_eps,
                     void* ws, size_t ws_bytes, void* stream);

/* The same row MLP on the fused BF16 path (tcgen05 GEMMs with BF16 operands
 * and FP32 accumulation, FP32 bias / ELU / LayerNorm, activations recomputed
 * in the backward). Covered shapes, H in {16, 32, 64}:
 *   encoder: dims[0] <= 16, every other width H, with LayerNorm;
 *   decoder: dims[0] = H, hidden widths H, dims[n_lin] <= 16, no LayerNorm;
 * and at H = 128 the encoder with 2 to 4 Linear layers, whose backward runs
 * one Linear at a time over chunks of 128-row tiles with the recomputed
 * activations in the workspace (Y and dY then 16-byte aligned, else GNN_EINVAL).
 * Same arguments and results as gnn_mlp_forward / gnn_mlp_backward (to BF16
 * tolerance); the forward needs no workspace, the backward the size reported
 * here for n_rows (per-CTA gradient partials; at H = 128 also the scratch of
 * up to 2^22 rows, and a smaller workspace down to one tile's scratch is
 * accepted and runs in more chunks, GNN_ENOMEM below that). GNN_EUNSUPPORTED
 * for other shapes (use the FP32 calls). */
int gnn_mlp_workspace_size_bf16(const gnn_mlp* P, int64_t n_rows, size_t* fwd_bytes, size_t* bwd_bytes);
int gnn_mlp_forward_bf16(const gnn_mlp* P, int64_t n_rows, const float* X, void* Y, int32_t y_bf16,
                         float ln_eps, void* ws, size_t ws_bytes, void* stream);
int gnn_mlp_backward_bf16(const gnn_mlp* P, int64_t n_rows, const float* X, const void* dY,
                          int32_t dy_bf16, float* dX, const gnn_mlp* dP, float ln_eps,
                          void* ws, size_t ws_bytes, void* stream);
/* Training with saved activations, as gnn_mp_forward_act: the forward also
 * writes the hidden activations h_0 .. h_{L-2} (BF16, block k of R =
 * ceil(n_rows / 128) * 128 rows of H, row k * R + r) to act, and the backward
 * given that act recomputes only the last Linear. act: device, 16-byte
 * aligned, of gnn_mlp_act_size_bf16 bytes, caller-owned and unchanged from the
 * forward to the backward; 0 bytes (act may be NULL: the plain calls) for
 * shapes outside the fused row MLP, the H = 128 encoder (which recomputes)
 * or (L - 1) * R >= 2^31. Same results as
 * gnn_mlp_forward_bf16 / gnn_mlp_backward_bf16. */
int gnn_mlp_act_size_bf16(const gnn_mlp* P, int64_t n_rows, size_t* bytes);
int gnn_mlp_forward_bf16_act(const gnn_mlp* P, int64_t n_rows, const float* X, void* Y, int32_t y_bf16,
                             float ln_eps, void* act, void* stream);
int gnn_mlp_backward_bf16_act(const gnn_mlp* P, int64_t n_rows, const float* X, const void* dY,
                              int32_t dy_bf16, float* dX, const gnn_mlp* dP, float ln_eps,
                              const void* act, void* ws, size_t ws_bytes, void* stream);

/* Consistent MSE loss, Eq. 8a-8c: L = sum_rows sum_f (1/d_i)(y - t)^2 /
 * (N_eff * F) with N_eff = sum_rows 1/d_i. y, t: device FP32 [n_rows x F].
 * loss: device FP32 scalar (written). dy: device FP32 [n_rows x F] = dL/dy,
 * or NULL. Reductions run in a fixed order (deterministic). ws >= 16 KiB. */
int gnn_consistent_loss(const gnn_graph_dev* G, const float* y, const float* t, int32_t F,
                        float* loss, float* dy, void* ws, size_t ws_bytes, void* stream);

/* ====================================================== kernel timing
 * Benchmark support (the paper has no counterpart). Between gnn_profile_start
 * and gnn_profile_stop every libgnnmp kernel launch is bracketed by a pair of
 * CUDA events on its stream (up to `capacity` launches; later launches are
 * not timed and the report says so). gnn_profile_report waits for the events
 * and writes one text line per kernel name, "<name> <launches> <total_ms>\n",
 * into out (host, `bytes` long, GNN_ENOMEM if too short). */
int gnn_profile_start(int32_t capacity);
int gnn_profile_stop(void);
int gnn_profile_report(char* out, size_t bytes);

/* ====================================================== diagnostics
 * The paper has no counterpart to these calls.
 *
 * gnn_measure_fp32_fma: the current device's FP32 FMA throughput, measured
 * with the library's own FMA kernel (independent chains of fused multiply-adds
 * per thread, two blocks of 1024 threads per SM, best of three CUDA-event timed
 * launches after one warm-up), in TFLOP/s at 2 FLOPs per FMA, and its SM count.
 * It is the peak the plain FP32 SIMT path is measured against. Synchronous on
 * `stream`; allocates nothing.
 *
 * gnn_selftest_bounded_wait: launches one warp that waits on an mbarrier no
 * thread ever arrives at, with the same bounded wait every libgnnmp kernel
 * uses but a limit of limit_ns (1 us .. 1 s) instead of the kernels' 1 s. The
 * wait gives up, latches the timeout in the device error word and the kernel
 * returns; *status (device int32) is then 1 (2 would mean the wait completed).
 * The next gnn_check returns GNN_ETIMEOUT and clears the word; the context stays
 * usable. Asynchronous on `stream`. */
int gnn_measure_fp32_fma(double* tflops, int32_t* sm_count, void* stream);
int gnn_selftest_bounded_wait(uint64_t limit_ns, int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GNNMP_H */
