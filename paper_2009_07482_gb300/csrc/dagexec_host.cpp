// dagexec_host.cpp -- host planner and C ABI of libdagexec.
//
// dag_create turns the paper's application DAG (§3) into a device plan:
//   1. validation: ids, shapes, dtypes, one writer per element, no in-place
//      kernel, acyclic kernel graph (Kahn's algorithm, smallest id first);
//   2. tiling: every kernel's output split into tiles (GEMM 128 x BN on the
//      tensor cores for bf16, BM x BN SIMT for f32; softmax row blocks;
//      elementwise row blocks);
//   3. dependency counters: one u32 per (written buffer, row block); a tile
//      increments the blocks it writes and waits until the blocks it reads
//      reach their writer-tile count.  This is the paper's command-queue
//      precedence E_Q (Def. 4 and rules i-iii after it) lifted from whole
//      kernels to tiles;
//   4. ordering: list scheduling of the tile graph on `grid` identical
//      workers, ready tiles ranked by the bottom-level rank of their kernel
//      (§5, clustering: the priority queue F ordered by bottom-level rank;
//      HEFT's upward rank).  The result is a linear extension of the tile
//      graph, which the persistent kernel's deadlock-freedom relies on;
//   5. device memory, TMA tensor maps and the kernel parameter block.
#include <cudaTypedefs.h>

#include <algorithm>
#include <tuple>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <queue>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "dag_internal.h"
#include "dagexec.h"

using namespace dagx;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static dag_status fail(dag_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return fail(DAG_EDEVICE, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char *dag_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// peaks for the time model and the roofline estimates
// ---------------------------------------------------------------------------
static double g_bf16_tflops = 1918.4, g_f32_tflops = 60.0, g_hbm_gbs = 6695.2;
// f32 on the tensor cores: tf32 runs at the nominal tf32 / bf16 ratio
// (1.1 / 2.25 PFLOP/s dense) of the bf16 peak, and a 3 x TF32 product takes three
static double tf32x3_tflops() { return g_bf16_tflops * (1.1 / 2.25) / 3.0; }

extern "C" void dag_set_peaks(double bf16_tflops, double f32_tflops, double hbm_gbs) {
  if (bf16_tflops > 0) g_bf16_tflops = bf16_tflops;
  if (f32_tflops > 0) g_f32_tflops = f32_tflops;
  if (hbm_gbs > 0) g_hbm_gbs = hbm_gbs;
}

// ---------------------------------------------------------------------------
// driver entry points (no link-time dependency on libcuda)
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 p_encode_tiled = nullptr;
static PFN_cuStreamWriteValue32_v11070 p_write_value32 = nullptr;
static std::once_flag g_driver_once;
static std::string g_driver_err;
static std::mutex g_prepared_mu;
static std::set<int> g_prepared;  // device ordinals whose executor attributes are set

static dag_status init_driver() {
  std::call_once(g_driver_once, [] {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void **)&p_encode_tiled, 12000,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p_encode_tiled)
      g_driver_err = "cuTensorMapEncodeTiled not available";
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", (void **)&p_write_value32, 11070,
                                         cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p_write_value32)
      g_driver_err = "cuStreamWriteValue32 not available";
  });
  if (!g_driver_err.empty()) return fail(DAG_EDEVICE, "%s", g_driver_err.c_str());
  // the executor's shared-memory attribute is set per device context: once
  // for every device this process plans on, with that device current
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return fail(DAG_EDEVICE, "no current CUDA device");
  std::lock_guard<std::mutex> lock(g_prepared_mu);
  if (!g_prepared.count(dev)) {
    if (exec_prepare() != cudaSuccess) return fail(DAG_EDEVICE, "cudaFuncSetAttribute failed on device %d", dev);
    g_prepared.insert(dev);
  }
  return DAG_OK;
}

// ---------------------------------------------------------------------------
// graph model
// ---------------------------------------------------------------------------
static inline int esize(int dt) { return dt == DAG_BF16 ? 2 : 4; }

struct Region {  // rows [r0,r1) x cols [c0,c1) of a root buffer
  int root, r0, r1, c0, c1;
};
static inline bool overlaps(const Region &a, const Region &b) {
  return a.root == b.root && a.r0 < b.r1 && b.r0 < a.r1 && a.c0 < b.c1 && b.c0 < a.c1;
}

struct Graph {
  int nb = 0, nn = 0;
  std::vector<dag_buffer_desc> bufs;
  std::vector<dag_node_desc> nodes;
  std::vector<int> root, coff;           // per buffer
  std::vector<std::vector<int>> succ, pred;
  std::vector<int> topo, topo_pos;
  std::vector<int> M, N, K;              // per node: per-batch GEMM dims, or rows/cols

  Region full(int b) const {
    return Region{root[b], 0, bufs[b].rows, coff[b], coff[b] + bufs[b].cols};
  }
  int inputs(int v, int out[3]) const {
    int k = 0;
    const dag_node_desc &n = nodes[v];
    out[k++] = n.a;
    if (n.op == DAG_OP_GEMM || n.op == DAG_OP_ADD) out[k++] = n.b;
    if (n.op == DAG_OP_GEMM && n.bias >= 0) out[k++] = n.bias;
    return k;
  }
};

static dag_status build_graph(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                              const dag_buffer_desc *buffers, int n_buffers, Graph &g) {
  if (n_nodes < 0 || n_buffers < 0 || n_edges < 0) return fail(DAG_EINVAL, "negative count");
  if ((n_nodes && !nodes) || (n_buffers && !buffers) || (n_edges && !edges))
    return fail(DAG_EINVAL, "null array with a nonzero count");
  g.nb = n_buffers;
  g.nn = n_nodes;
  g.bufs.assign(buffers, buffers + n_buffers);
  g.nodes.assign(nodes, nodes + n_nodes);
  g.root.resize(n_buffers);
  g.coff.resize(n_buffers);
  auto valid = [&](int id) { return id >= 0 && id < n_buffers; };
  for (int i = 0; i < n_buffers; ++i) {
    const dag_buffer_desc &b = buffers[i];
    if (b.rows <= 0 || b.cols <= 0) return fail(DAG_ESHAPE, "buffer %d: shape %dx%d", i, b.rows, b.cols);
    if (b.dtype != DAG_F32 && b.dtype != DAG_BF16) return fail(DAG_EDTYPE, "buffer %d: dtype %d", i, b.dtype);
    if (b.flags & ~7u) return fail(DAG_EINVAL, "buffer %d: unknown flags", i);
    if ((b.flags & DAG_BUF_RESIDENT) && !(b.flags & DAG_BUF_INPUT))
      return fail(DAG_EINVAL, "buffer %d: RESIDENT without INPUT", i);
    g.root[i] = i;
    g.coff[i] = 0;
    if (b.view_of >= 0) {
      if (!valid(b.view_of) || b.view_of == i) return fail(DAG_EINVAL, "buffer %d: bad view parent", i);
      const dag_buffer_desc &p = buffers[b.view_of];
      if (p.view_of >= 0) return fail(DAG_EINVAL, "buffer %d: view of a view", i);
      if (p.rows != b.rows || b.col_offset < 0 || b.col_offset + b.cols > p.cols)
        return fail(DAG_ESHAPE, "buffer %d: view does not fit its parent", i);
      if (p.dtype != b.dtype) return fail(DAG_EDTYPE, "buffer %d: view dtype differs from parent", i);
      if (b.flags) return fail(DAG_EINVAL, "buffer %d: a view cannot carry INPUT/OUTPUT flags", i);
      g.root[i] = b.view_of;
      g.coff[i] = b.col_offset;
    }
  }
  g.M.assign(n_nodes, 0);
  g.N.assign(n_nodes, 0);
  g.K.assign(n_nodes, 0);
  for (int v = 0; v < n_nodes; ++v) {
    const dag_node_desc &n = nodes[v];
    if (!valid(n.a) || !valid(n.out)) return fail(DAG_EINVAL, "node %d: bad buffer id", v);
    if (n.act < DAG_ACT_NONE || n.act > DAG_ACT_GELU) return fail(DAG_EINVAL, "node %d: bad activation", v);
    const dag_buffer_desc &A = buffers[n.a], &O = buffers[n.out];
    if (g.bufs[g.root[n.out]].flags & DAG_BUF_INPUT)
      return fail(DAG_EMULTIWRITER, "node %d writes input buffer %d", v, n.out);
    switch (n.op) {
      case DAG_OP_GEMM: {
        if (!valid(n.b)) return fail(DAG_EINVAL, "node %d: bad B id", v);
        if (n.batch < 1) return fail(DAG_EINVAL, "node %d: batch %d", v, n.batch);
        const dag_buffer_desc &B = buffers[n.b];
        if (A.rows % n.batch || B.rows % n.batch) return fail(DAG_ESHAPE, "node %d: batch does not divide rows", v);
        const int M = A.rows / n.batch, K = A.cols;
        const int N = n.trans_b ? B.rows / n.batch : B.cols;
        const int Kb = n.trans_b ? B.cols : B.rows / n.batch;
        if (Kb != K) return fail(DAG_ESHAPE, "node %d: inner dims %d vs %d", v, K, Kb);
        if (O.rows != A.rows || O.cols != N) return fail(DAG_ESHAPE, "node %d: output %dx%d, want %dx%d", v, O.rows, O.cols, A.rows, N);
        if (A.dtype != B.dtype) return fail(DAG_EDTYPE, "node %d: A and B dtypes differ", v);
        if (n.bias >= 0) {
          if (!valid(n.bias)) return fail(DAG_EINVAL, "node %d: bad bias id", v);
          if (buffers[n.bias].rows != 1 || buffers[n.bias].cols != N) return fail(DAG_ESHAPE, "node %d: bias shape", v);
        }
        g.M[v] = M; g.N[v] = N; g.K[v] = K;
        break;
      }
      case DAG_OP_ADD:
        if (!valid(n.b)) return fail(DAG_EINVAL, "node %d: bad B id", v);
        if (buffers[n.b].rows != O.rows || buffers[n.b].cols != O.cols || A.rows != O.rows || A.cols != O.cols)
          return fail(DAG_ESHAPE, "node %d: add shapes", v);
        g.M[v] = O.rows; g.N[v] = O.cols; g.K[v] = 0;
        break;
      case DAG_OP_SOFTMAX:
      case DAG_OP_UNARY:
        if (A.rows != O.rows || A.cols != O.cols) return fail(DAG_ESHAPE, "node %d: shapes", v);
        g.M[v] = O.rows; g.N[v] = O.cols; g.K[v] = 0;
        break;
      default:
        return fail(DAG_EINVAL, "node %d: unknown op %d", v, n.op);
    }
  }
  // writers indexed by root buffer: one writer per element, no in-place kernel
  std::vector<std::vector<int>> writers(n_buffers);
  for (int u = 0; u < n_nodes; ++u) writers[g.root[nodes[u].out]].push_back(u);
  for (int r = 0; r < n_buffers; ++r) {
    std::vector<std::pair<int, int>> iv;  // (c0, node) sorted by first column
    for (int u : writers[r]) iv.push_back({g.full(nodes[u].out).c0, u});
    std::sort(iv.begin(), iv.end());
    for (size_t i = 1; i < iv.size(); ++i) {
      const Region a = g.full(nodes[iv[i - 1].second].out), b = g.full(nodes[iv[i].second].out);
      if (overlaps(a, b))
        return fail(DAG_EMULTIWRITER, "nodes %d and %d write overlapping buffers", iv[i - 1].second, iv[i].second);
    }
  }
  for (int u = 0; u < n_nodes; ++u) {
    const Region wu = g.full(nodes[u].out);
    int in[3];
    const int k = g.inputs(u, in);
    for (int q = 0; q < k; ++q)
      if (overlaps(wu, g.full(in[q]))) return fail(DAG_EMULTIWRITER, "node %d reads what it writes", u);
  }
  // kernel graph: u -> v when v reads a region u writes
  g.succ.assign(n_nodes, {});
  g.pred.assign(n_nodes, {});
  for (int v = 0; v < n_nodes; ++v) {
    int in[3];
    const int k = g.inputs(v, in);
    for (int q = 0; q < k; ++q) {
      const Region r = g.full(in[q]);
      for (int u : writers[r.root]) {
        if (u == v || !overlaps(g.full(nodes[u].out), r)) continue;
        if (std::find(g.pred[v].begin(), g.pred[v].end(), u) == g.pred[v].end()) {
          g.pred[v].push_back(u);
          g.succ[u].push_back(v);
        }
      }
      // every element read must be written by some kernel or be an input
      if (g.bufs[r.root].flags & DAG_BUF_INPUT) continue;
      std::vector<std::pair<int, int>> cov;
      for (int u : writers[r.root]) {
        const Region w = g.full(nodes[u].out);
        cov.push_back({w.c0, w.c1});
      }
      std::sort(cov.begin(), cov.end());
      int reach = r.c0;
      for (auto &c : cov)
        if (c.first <= reach) reach = std::max(reach, c.second);
      if (reach < r.c1) return fail(DAG_EINVAL, "node %d reads buffer %d, which is neither an input nor fully written", v, in[q]);
    }
  }
  for (int v = 0; v < n_nodes; ++v) {
    std::sort(g.succ[v].begin(), g.succ[v].end());
    std::sort(g.pred[v].begin(), g.pred[v].end());
  }
  // edges given by the caller must be implied by the buffers
  for (int e = 0; e < n_edges; ++e) {
    const dag_edge &E = edges[e];
    if (E.src_node < 0 || E.src_node >= n_nodes || E.dst_node < 0 || E.dst_node >= n_nodes || !valid(E.src_buf) ||
        !valid(E.dst_buf))
      return fail(DAG_EINVAL, "edge %d: bad id", e);
    if (nodes[E.src_node].out != E.src_buf) return fail(DAG_EINVAL, "edge %d: node %d does not write buffer %d", e, E.src_node, E.src_buf);
    int in[3];
    const int k = g.inputs(E.dst_node, in);
    bool reads = false;
    for (int q = 0; q < k; ++q) reads |= in[q] == E.dst_buf;
    if (!reads) return fail(DAG_EINVAL, "edge %d: node %d does not read buffer %d", e, E.dst_node, E.dst_buf);
    if (!overlaps(g.full(E.src_buf), g.full(E.dst_buf))) return fail(DAG_EINVAL, "edge %d: buffers do not overlap", e);
  }
  // Kahn, smallest id first
  std::vector<int> indeg(n_nodes, 0);
  for (int v = 0; v < n_nodes; ++v) indeg[v] = (int)g.pred[v].size();
  std::priority_queue<int, std::vector<int>, std::greater<int>> ready;
  for (int v = 0; v < n_nodes; ++v)
    if (!indeg[v]) ready.push(v);
  g.topo.clear();
  while (!ready.empty()) {
    const int u = ready.top();
    ready.pop();
    g.topo.push_back(u);
    for (int v : g.succ[u])
      if (--indeg[v] == 0) ready.push(v);
  }
  if ((int)g.topo.size() != n_nodes) return fail(DAG_ECYCLE, "the kernel graph has a cycle");
  g.topo_pos.assign(n_nodes, 0);
  for (int i = 0; i < n_nodes; ++i) g.topo_pos[g.topo[i]] = i;
  return DAG_OK;
}

// ---------------------------------------------------------------------------
// dag_analyze: §3 Defs. 1-3 and the copy / edge classification
// ---------------------------------------------------------------------------
extern "C" dag_status dag_analyze(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                                  const dag_buffer_desc *buffers, int n_buffers, dag_analysis *out) {
  if (!out) return fail(DAG_EINVAL, "null output");
  Graph g;
  dag_status s = build_graph(nodes, n_nodes, edges, n_edges, buffers, n_buffers, g);
  if (s) return s;
  out->n_nodes = n_nodes;
  out->n_copies = 0;
  out->n_edge_cls = 0;
  for (int v = 0; v < n_nodes; ++v) {
    // FRONT(T): no input produced inside T (every producer, if any, lies in another component)
    // END(T):   no output consumed inside T
    bool front = true, end = true;
    for (int u : g.pred[v])
      if (nodes[u].component == nodes[v].component) front = false;
    for (int w : g.succ[v])
      if (nodes[w].component == nodes[v].component) end = false;
    int c = (front ? 1 : 0) | (end ? 2 : 0);
    if (!front && !end) c |= 4;  // IN(T)
    if (out->cls) out->cls[v] = c;
    if (out->topo) out->topo[v] = g.topo[v];
  }
  auto add_copy = [&](int node, int buf, int is_write, int isolated) {
    if (out->copies && out->n_copies < out->cap_copies)
      out->copies[out->n_copies] = dag_copy_class{node, buf, is_write, isolated};
    out->n_copies++;
  };
  for (int v = 0; v < n_nodes; ++v) {
    int in[3];
    const int k = g.inputs(v, in);
    for (int q = 0; q < k; ++q) {
      bool produced = false;
      for (int u : g.pred[v]) produced |= overlaps(g.full(nodes[u].out), g.full(in[q]));
      add_copy(v, in[q], 1, produced ? 0 : 1);  // (b,k) in E_I: isolated write iff no (b',b) in E
    }
    bool consumed = !g.succ[v].empty();
    add_copy(v, nodes[v].out, 0, consumed ? 0 : 1);  // (k,b) in E_O: isolated read iff no (b,b') in E
  }
  for (int u = 0; u < n_nodes; ++u)
    for (int v : g.succ[u]) {
      int in[3];
      const int k = g.inputs(v, in);
      for (int q = 0; q < k; ++q) {
        if (!overlaps(g.full(nodes[u].out), g.full(in[q]))) continue;
        if (out->edge_cls && out->n_edge_cls < out->cap_edges)
          out->edge_cls[out->n_edge_cls] =
              dag_edge_class{u, nodes[u].out, v, in[q], nodes[u].component != nodes[v].component ? 1 : 0};
        out->n_edge_cls++;
      }
    }
  return DAG_OK;
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct Plan {
  Graph g;
  dag_options opt{};
  int n_sm = 148, grid = 148;
  std::vector<int> cfg;                 // per node tile config
  std::vector<char> tf32;               // per node: f32 GEMM on the tensor cores (3 x TF32)
  std::vector<char> tf32w;              // per node: ... in the wide form (128 x 128 / 256, B K-major)
  std::vector<int> nsplit;              // per node: split-K factor S (0 = none)
  std::vector<char> store_t;            // per buffer: a weight kept transposed on the device (layout.cu)
  std::vector<int> t_batch, t_K, t_N;   // its per-batch shape as given (K x N)
  bool allow_layout = true;             // not for caller-owned buffers (the no-alloc entry point)
  std::vector<int> absorbed_by;         // per node: the GEMM whose epilogue computes it, or -1
  std::vector<int> merged_into;         // per node: the sibling GEMM whose tiles compute it as a column
                                        // slice of a merged GEMM (itself for that GEMM), or -1
  std::vector<int> merge_coff;          // per node of a merged group: its first column in the merged GEMM
  bool merged_done = false;             // the graph's sibling GEMMs have been merged (once per plan)
  std::vector<char> merge_parent;       // per buffer: a parent made for merged siblings' slices
  std::vector<dag_node_desc> orig_nodes;  // the kernels as given (empty: no merge), for the DAG's own
  std::vector<int> orig_N;                // algorithmic work and roofline
  std::vector<std::vector<int>> post;   // per GEMM: elementwise kernels fused into its epilogue, in order
  bool allow_split = true;              // split K needs scratch memory (not in the no-alloc entry point)
  std::vector<TileDesc> tiles;          // node-major creation order
  std::vector<int> node_first, node_count;
  std::vector<TileDesc> queue;          // queue order (persistent mode)
  std::vector<int> queue_src;           // queue position -> creation index
  std::vector<Wait> waits;
  std::vector<uint32_t> rels;
  int n_counters = 0;
  std::vector<int> flag_of_root;        // streamed-input flag index, or -1
  int n_flags = 0;
  std::vector<double> rank;             // per node bottom-level rank (us)
  std::vector<double> node_cost;        // per node estimated time (us)
  double flops = 0, bytes = 0, cp_us = 0, work_us = 0;
};

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// the buffer kernel v's tiles write: a GEMM with fused kernels writes the last one's output
static int tile_out(const Plan &P, int v) {
  return P.post.empty() || P.post[v].empty() ? P.g.nodes[v].out : P.g.nodes[P.post[v].back()].out;
}

// per-tile time model (us): roofline of the tile's work on one SM plus a
// fixed per-tile overhead
static double tile_time_us(const Plan &P, int v, const TileDesc &t) {
  const Graph &g = P.g;
  const dag_node_desc &n = g.nodes[v];
  const double per_sm_bw = g_hbm_gbs * 1e9 / P.n_sm * 2.0;  // an SM alone streams faster than its fair share
  const double rows = t.r1 - t.r0, cols = t.c1 - t.c0;
  if (n.op == DAG_OP_GEMM) {
    const double K = (double)g.K[v] / (t.split ? split_count(t) : 1);
    const double flops = 2.0 * rows * cols * K;
    const int ea = esize(g.bufs[n.a].dtype);
    const double bytes = (rows + cols) * K * ea + rows * cols * esize(g.bufs[n.out].dtype);
    double rate;
    if (t.op == T_GEMM_BF16) {
      const double eff = t.cfg >= 256 ? 0.8 : t.cfg >= 128 ? 0.7 : 0.5;
      rate = g_bf16_tflops * 1e12 / P.n_sm * eff;
    } else if (t.op == T_GEMM_TF32) {
      // three tf32 MMAs (half the bf16 rate) per product, 128 x 64 tiles
      rate = g_bf16_tflops * 1e12 / P.n_sm / 6.0 * 0.5;
    } else if (t.op == T_GEMM_TF32W) {
      rate = g_bf16_tflops * 1e12 / P.n_sm / 6.0 * (t.cfg >= 256 ? 0.8 : 0.65);
    } else {
      rate = g_f32_tflops * 1e12 / P.n_sm * 0.6;
    }
    return std::max(flops / rate, bytes / per_sm_bw) * 1e6 + 1.0;
  }
  double bytes = rows * cols * (esize(g.bufs[n.a].dtype) + esize(g.bufs[n.out].dtype));
  if (n.op == DAG_OP_ADD) bytes += rows * cols * esize(g.bufs[n.b].dtype);
  return bytes / per_sm_bw * 1e6 + 0.7;
}

static int ntiles_gemm(const Graph &g, int v, int bm, int bn) {
  return g.nodes[v].batch * ((g.M[v] + bm - 1) / bm) * ((g.N[v] + bn - 1) / bn);
}

// a node whose tiles another (merged) GEMM computes
static inline bool merged_away(const Plan &P, int v) {
  return !P.merged_into.empty() && P.merged_into[v] >= 0 && P.merged_into[v] != v;
}

// Sibling GEMMs merged by column slices (dag_options.merge = 0).  GEMMs of
// one task component that read the same A with trans_b = 0, batch 1, one K,
// activation and scale, each with a resident weight (and all or none with a
// resident bias) that no other kernel reads and that no view covers, and with
// a private intermediate output that no view covers, each narrower than 256
// columns in 16-byte slices: their weights, biases and outputs become
// column-slice views of three new parent buffers, and the first of them in
// topological order computes the parent GEMM over the summed width.  A
// tcgen05.mma of M = 128 takes 128 clocks for any N up to 128 and 166 for N
// = 256, so N = 64 kernels run their tensor cores at a third of the rate that
// one wide GEMM reaches.  Every output element is the same dot product in the
// same K order, so the results are bit-identical; the dependency counters,
// kept per root row block, see the views as they see every view.  The
// merged GEMM inherits the successors of all its siblings (Alg. 1's task
// components keep their order), and the siblings keep no tiles of their own.
// A buffer id of the caller's description (not a parent the planner added
// for merged siblings): the only ids the public calls accept.
static bool caller_buf(const Plan &P, int b) {
  return b >= 0 && b < P.g.nb && !(b < (int)P.merge_parent.size() && P.merge_parent[b]);
}

static void choose_merges(Plan &P) {
  if (P.merged_done) return;
  P.merged_done = true;
  Graph &g = P.g;
  P.merged_into.assign(g.nn, -1);
  P.merge_coff.assign(g.nn, 0);
  P.merge_parent.assign(g.nb, 0);
  if (!P.allow_layout || P.opt.keep_layout || P.opt.merge == 1) return;
  const int nb0 = g.nb;
  std::vector<int> readers(nb0, 0);
  std::vector<char> viewed(nb0, 0);
  for (int b = 0; b < nb0; ++b)
    if (g.bufs[b].view_of >= 0) viewed[g.root[b]] = 1;
  for (int v = 0; v < g.nn; ++v) {
    int in[3];
    const int k = g.inputs(v, in);
    for (int q = 0; q < k; ++q) readers[in[q]]++;
  }
  const uint32_t res = DAG_BUF_INPUT | DAG_BUF_RESIDENT;
  auto private_weight = [&](int b) {
    const dag_buffer_desc &d = g.bufs[b];
    return d.view_of < 0 && !viewed[b] && readers[b] == 1 && (d.flags & (res | DAG_BUF_OUTPUT)) == res;
  };
  struct Cand {
    int a, comp, K, M, act, bdt, odt, bias, biasdt;
    uint32_t scale;
    int pos, v;
  };
  std::vector<Cand> c;
  for (int v = 0; v < g.nn; ++v) {
    const dag_node_desc &n = g.nodes[v];
    if (n.op != DAG_OP_GEMM || n.batch != 1 || n.trans_b || g.N[v] >= 256) continue;
    const dag_buffer_desc &O = g.bufs[n.out];
    const int ob = esize(O.dtype), bb = esize(g.bufs[n.b].dtype);
    if (!private_weight(n.b) || (n.bias >= 0 && !private_weight(n.bias))) continue;
    if (O.view_of >= 0 || viewed[n.out] || (O.flags & (DAG_BUF_INPUT | DAG_BUF_OUTPUT))) continue;
    if ((g.N[v] * ob) % 16 || (g.N[v] * bb) % 16) continue;
    uint32_t sc;
    memcpy(&sc, &n.scale, 4);
    c.push_back(Cand{n.a, n.component, g.K[v], g.M[v], n.act, g.bufs[n.b].dtype, O.dtype, n.bias >= 0,
                     n.bias >= 0 ? g.bufs[n.bias].dtype : -1, sc, g.topo_pos[v], v});
  }
  auto key = [](const Cand &x) {
    return std::make_tuple(x.a, x.comp, x.K, x.M, x.act, x.bdt, x.odt, x.bias, x.biasdt, x.scale);
  };
  std::sort(c.begin(), c.end(), [&](const Cand &x, const Cand &y) {
    return key(x) != key(y) ? key(x) < key(y) : x.pos < y.pos;
  });
  auto add_buf = [&](int rows, int cols, int dtype, uint32_t flags) {
    dag_buffer_desc d{};
    d.rows = rows;
    d.cols = cols;
    d.dtype = dtype;
    d.flags = flags;
    d.view_of = -1;
    d.col_offset = 0;
    g.bufs.push_back(d);
    g.root.push_back(g.nb);
    g.coff.push_back(0);
    P.merge_parent.push_back(1);
    return g.nb++;
  };
  auto make_view = [&](int b, int parent, int off) {
    g.bufs[b].view_of = parent;
    g.bufs[b].col_offset = off;
    g.root[b] = parent;
    g.coff[b] = off;
  };
  for (size_t i = 0; i < c.size();) {
    size_t j = i + 1;
    while (j < c.size() && key(c[j]) == key(c[i])) ++j;
    if (j - i >= 2) {
      if (P.orig_nodes.empty()) {
        P.orig_nodes = g.nodes;
        P.orig_N = g.N;
      }
      const int L = c[i].v;  // the first in topological order computes the group
      int total = 0;
      for (size_t q = i; q < j; ++q) total += g.N[c[q].v];
      const int Bp = add_buf(g.K[L], total, c[i].bdt, res);
      const int Op = add_buf(g.M[L], total, c[i].odt, 0);
      const int Cp = c[i].bias ? add_buf(1, total, c[i].biasdt, res) : -1;
      int off = 0;
      std::vector<int> succ;
      for (size_t q = i; q < j; ++q) {
        const int v = c[q].v;
        const dag_node_desc &n = g.nodes[v];
        make_view(n.b, Bp, off);
        make_view(n.out, Op, off);
        if (Cp >= 0) make_view(n.bias, Cp, off);
        P.merged_into[v] = L;
        P.merge_coff[v] = off;
        off += g.N[v];
        succ.insert(succ.end(), g.succ[v].begin(), g.succ[v].end());
      }
      dag_node_desc &ml = g.nodes[L];
      ml.b = Bp;
      ml.out = Op;
      ml.bias = Cp;
      g.N[L] = total;
      for (int w : succ)
        if (std::find(g.succ[L].begin(), g.succ[L].end(), w) == g.succ[L].end()) {
          g.succ[L].push_back(w);
          g.pred[w].push_back(L);
        }
      std::sort(g.succ[L].begin(), g.succ[L].end());
      for (int w : succ) std::sort(g.pred[w].begin(), g.pred[w].end());
    }
    i = j;
  }
}

// tile shapes: bf16 GEMMs take the widest BN (256/128/64) that still gives
// the kernel's concurrency level enough tiles to fill the GPU; f32 GEMMs
// likewise among 128x128 / 128x64 / 64x64.
static void choose_configs(Plan &P) {
  Graph &g = P.g;
  const int nn = g.nn;
  std::vector<int> depth(nn, 0);
  for (int u : g.topo)
    for (int v : g.succ[u]) depth[v] = std::max(depth[v], depth[u] + 1);
  int maxd = 0;
  for (int v = 0; v < nn; ++v) maxd = std::max(maxd, depth[v]);
  P.cfg.assign(nn, 0);
  P.tf32.assign(nn, 0);
  P.tf32w.assign(nn, 0);
  for (int v = 0; v < nn; ++v) {
    const dag_node_desc &n = g.nodes[v];
    if (n.op != DAG_OP_GEMM || g.bufs[n.a].dtype != DAG_F32 || P.opt.f32_gemm == DAG_F32_GEMM_SIMT) continue;
    // TMA operands: 16-byte aligned column views (roots and row pitches are)
    P.tf32[v] = ((size_t)g.coff[n.a] * 4) % 16 == 0 && ((size_t)g.coff[n.b] * 4) % 16 == 0;
    // the wide form reads B K-major (given so, or a weight kept transposed)
    // and pays off from 128 output columns on
    const bool kmajor = n.trans_b || P.store_t[g.root[n.b]];
    P.tf32w[v] = P.tf32[v] && kmajor && g.N[v] > kTf32BN && P.opt.f32_gemm != DAG_F32_GEMM_TENSOR_NARROW;
  }
  static const int bns[3] = {256, 128, 64};
  static const int wbns[3] = {256, 128, 128};
  static const int f32c[3][3] = {{F32_128x128, 128, 128}, {F32_128x64, 128, 64}, {F32_64x64, 64, 64}};
  for (int pass = 0; pass < 3; ++pass) {
    // concurrency of a depth level at option index `pass`
    std::vector<long> level(maxd + 1, 0);
    for (int v = 0; v < nn; ++v) {
      const dag_node_desc &n = g.nodes[v];
      if (merged_away(P, v)) continue;
      if (n.op != DAG_OP_GEMM) { level[depth[v]] += 8; continue; }
      if (P.tf32w[v]) level[depth[v]] += ntiles_gemm(g, v, 128, wbns[pass]);
      else if (P.tf32[v]) level[depth[v]] += ntiles_gemm(g, v, 128, kTf32BN);
      else if (g.bufs[n.a].dtype == DAG_BF16) level[depth[v]] += ntiles_gemm(g, v, 128, bns[pass]);
      else level[depth[v]] += ntiles_gemm(g, v, f32c[pass][1], f32c[pass][2]);
    }
    for (int v = 0; v < nn; ++v) {
      const dag_node_desc &n = g.nodes[v];
      if (n.op != DAG_OP_GEMM || P.cfg[v]) continue;
      const bool enough = level[depth[v]] >= P.n_sm * 3 / 4 || pass == 2;
      if (!enough) continue;
      if (P.tf32w[v] && pass == 2 && g.K[v] < 1024 && P.opt.f32_gemm != DAG_F32_GEMM_TENSOR_WIDE) {
        // a level too small for 128-column tiles and a short K loop (no
        // split): twice as many 128 x 64 tiles fill more SMs
        P.tf32w[v] = 0;
        P.cfg[v] = kTf32BN + 100;
      } else if (P.tf32w[v]) {
        int bn = wbns[pass];
        while (bn > 128 && bn / 2 >= round_up(g.N[v], 64)) bn /= 2;  // no wider than N
        P.cfg[v] = bn + 100;
      } else if (P.tf32[v]) {
        P.cfg[v] = kTf32BN + 100;
      } else if (g.bufs[n.a].dtype == DAG_BF16) {
        int bn = bns[pass];
        while (bn > 64 && bn / 2 >= round_up(g.N[v], 64)) bn /= 2;  // no wider than N
        P.cfg[v] = bn;
      } else {
        P.cfg[v] = f32c[pass][0] + 100;  // +100 marks "set"
      }
    }
  }
  for (int v = 0; v < nn; ++v) {
    const dag_node_desc &n = g.nodes[v];
    if (n.op != DAG_OP_GEMM) continue;
    if (g.bufs[n.a].dtype == DAG_BF16) {
      if (P.opt.tile_override == 64 || P.opt.tile_override == 128 || P.opt.tile_override == 256)
        P.cfg[v] = P.opt.tile_override;
    } else {
      P.cfg[v] -= 100;
      // an f32 GEMM that can take the wide form: 128 / 256 forces that width, 64 the 128 x 64 form
      const bool can_wide = P.tf32[v] && (n.trans_b || P.store_t[g.root[n.b]]) && g.N[v] > kTf32BN &&
                            P.opt.f32_gemm != DAG_F32_GEMM_TENSOR_NARROW;
      if (can_wide && (P.opt.tile_override == 128 || P.opt.tile_override == 256)) {
        P.tf32w[v] = 1;
        P.cfg[v] = P.opt.tile_override;
      } else if (can_wide && P.opt.tile_override == 64) {
        P.tf32w[v] = 0;
        P.cfg[v] = kTf32BN;
      }
    }
  }
}

// Weights kept K-major on the device: a resident bf16/f32 input buffer that
// every reader takes as the B operand of a GEMM with trans_b = 0, all with
// one (batch, K, N), with no views into it.  The GEMMs then run as trans_b =
// 1 over the transposed copy (see layout.cu).
static void choose_layouts(Plan &P) {
  Graph &g = P.g;
  P.store_t.assign(g.nb, 0);
  P.t_batch.assign(g.nb, 0);
  P.t_K.assign(g.nb, 0);
  P.t_N.assign(g.nb, 0);
  if (!P.allow_layout || P.opt.keep_layout) return;
  std::vector<char> ok(g.nb, 1);
  for (int b = 0; b < g.nb; ++b)  // read through a view (the slices of merged siblings' weights aside:
    if (g.root[b] != b && !P.merge_parent[g.root[b]]) ok[g.root[b]] = 0;  // uploaded slice by slice)
  std::vector<int> readers(g.nb, 0);
  for (int v = 0; v < g.nn; ++v) {
    if (merged_away(P, v)) continue;
    const dag_node_desc &n = g.nodes[v];
    int in[3];
    const int k = g.inputs(v, in);
    for (int q = 0; q < k; ++q) {
      const int r = g.root[in[q]];
      readers[r]++;
      if (n.op != DAG_OP_GEMM || q != 1 || n.trans_b || in[0] == in[1] || (k > 2 && in[2] == in[1])) {
        ok[r] = 0;
        continue;
      }
      if (readers[r] == 1) {
        P.t_batch[r] = n.batch; P.t_K[r] = g.K[v]; P.t_N[r] = g.N[v];
      } else if (P.t_batch[r] != n.batch || P.t_K[r] != g.K[v] || P.t_N[r] != g.N[v]) {
        ok[r] = 0;
      }
    }
  }
  for (int b = 0; b < g.nb; ++b) {
    const dag_buffer_desc &d = g.bufs[b];
    const uint32_t want = DAG_BUF_INPUT | DAG_BUF_RESIDENT;
    P.store_t[b] = ok[b] && readers[b] > 0 && g.root[b] == b && (d.flags & want) == want &&
                   (d.dtype == DAG_BF16 || d.dtype == DAG_F32);
  }
}

// Epilogue fusion (DAG_FUSE_ACT, DAG_FUSE_ALL): an activation kernel (with
// DAG_FUSE_ALL also an add) reading the output O of a tensor-core GEMM runs
// inside that GEMM's epilogue when no other kernel reads O, O is a plain
// buffer (not a view, none into it) and neither a DAG input nor output, and
// the kernel is not fused elsewhere; its own output may continue the chain,
// up to kMaxPost kernels.  O is then never written: the epilogue rounds each
// step to the dtype of the buffer it stands for, so the values are those of
// the unfused DAG.  An add's other operand is waited for before the epilogue
// (a late wait), not before the K loop.
static void choose_fusion(Plan &P) {
  Graph &g = P.g;
  P.absorbed_by.assign(g.nn, -1);
  P.post.assign(g.nn, {});
  if (P.opt.fuse != DAG_FUSE_ACT && P.opt.fuse != DAG_FUSE_ALL) return;
  std::vector<int> views(g.nb, 0);
  for (int b = 0; b < g.nb; ++b)
    if (g.root[b] != b) views[g.root[b]]++;
  auto private_out = [&](int v) {  // read by exactly one kernel, and only by it
    const int o = g.nodes[v].out;
    return g.root[o] == o && !views[o] && !(g.bufs[o].flags & (DAG_BUF_INPUT | DAG_BUF_OUTPUT)) &&
           g.succ[v].size() == 1;
  };
  for (int v : g.topo) {
    const dag_node_desc &n = g.nodes[v];
    if (n.op != DAG_OP_GEMM || !(g.bufs[n.a].dtype == DAG_BF16 || P.tf32[v])) continue;
    int cur = v;
    while ((int)P.post[v].size() < kMaxPost && private_out(cur)) {
      const int e = g.succ[cur][0], o = g.nodes[cur].out;
      const dag_node_desc &m = g.nodes[e];
      if (P.absorbed_by[e] >= 0) break;
      if (m.op == DAG_OP_ADD) {
        if (P.opt.fuse != DAG_FUSE_ALL || (m.a == o) == (m.b == o)) break;  // reads O exactly once
      } else if (m.op != DAG_OP_UNARY || m.a != o) {
        break;
      }
      P.absorbed_by[e] = v;
      P.post[v].push_back(e);
      cur = e;
    }
  }
}

// Split K: a bf16 GEMM whose depth level leaves most SMs idle and whose K
// loop is long is cut into S partials of K/S each (S <= 4, at least 16 K
// blocks per partial), so that the level's tiles fill up to the SM count.
// The last partial of each output tile adds the others' partial sums in a
// fixed order, so the result does not depend on the schedule.
static void choose_split(Plan &P) {
  Graph &g = P.g;
  const int nn = g.nn;
  P.nsplit.assign(nn, 0);
  if (!P.allow_split || P.opt.split_k == 1) return;
  std::vector<int> depth(nn, 0);
  for (int u : g.topo)
    for (int v : g.succ[u]) depth[v] = std::max(depth[v], depth[u] + 1);
  std::vector<long> level(nn + 1, 0);
  for (int v = 0; v < nn; ++v) {
    const dag_node_desc &n = g.nodes[v];
    if (merged_away(P, v)) continue;
    if (n.op != DAG_OP_GEMM) {
      if (P.absorbed_by[v] < 0) level[depth[v]] += 8;
      continue;
    }
    const int bn = g.bufs[n.a].dtype == DAG_BF16 || P.tf32w[v] ? P.cfg[v] : 64;
    level[depth[v]] += ntiles_gemm(g, v, 128, std::max(bn, 64));
  }
  for (int v = 0; v < nn; ++v) {
    const dag_node_desc &n = g.nodes[v];
    if (n.op != DAG_OP_GEMM || merged_away(P, v)) continue;
    const long lt = level[depth[v]];
    int S = 0, kit = 0;
    if (g.bufs[n.a].dtype == DAG_BF16) {
      kit = (g.K[v] + kBK - 1) / kBK;
      if (lt * 2 > P.n_sm || kit < 32) continue;
      S = std::min({4, (int)(P.n_sm / std::max(1L, lt)), kit / 16});
    } else if (P.tf32w[v]) {
      // the wide f32 form: at least 16 stages (256 of K) per partial
      kit = (g.K[v] + kBKW - 1) / kBKW;
      if (lt * 2 > P.n_sm || kit < 32) continue;
      S = std::min({4, (int)(P.n_sm / std::max(1L, lt)), kit / 16});
    } else {
      continue;
    }
    // every partial gets a non-empty share of the K blocks
    while (S >= 2 && (long)(S - 1) * ((kit + S - 1) / S) >= kit) --S;
    if (S >= 2) P.nsplit[v] = S;
  }
}

// depth of every kernel in the kernel DAG (longest path from a root)
static std::vector<int> depths(const Graph &g) {
  std::vector<int> d(g.nn, 0);
  for (int u : g.topo)
    for (int v : g.succ[u]) d[v] = std::max(d[v], d[u] + 1);
  return d;
}

static void make_tiles(Plan &P) {
  Graph &g = P.g;
  P.tiles.clear();
  // memory-bound kernels at one depth level share the GPU: give each a share
  // of about two tiles per SM in proportion to its elements
  const std::vector<int> dep = depths(g);
  std::vector<double> level_elems(g.nn + 1, 0.0);
  for (int v = 0; v < g.nn; ++v)
    if (g.nodes[v].op != DAG_OP_GEMM && P.absorbed_by[v] < 0)
      level_elems[dep[v]] += (double)g.bufs[g.nodes[v].out].rows * g.bufs[g.nodes[v].out].cols;
  P.node_first.assign(g.nn, 0);
  P.node_count.assign(g.nn, 0);
  for (int v = 0; v < g.nn; ++v) {
    const dag_node_desc &n = g.nodes[v];
    P.node_first[v] = (int)P.tiles.size();
    auto push = [&](int op, int r0, int r1, int c0, int c1, int cfg) {
      TileDesc t{};
      t.node = v; t.op = op; t.r0 = r0; t.r1 = r1; t.c0 = c0; t.c1 = c1; t.cfg = cfg;
      P.tiles.push_back(t);
    };
    const int R = g.bufs[n.out].rows, C = g.bufs[n.out].cols;
    if (P.absorbed_by[v] >= 0 || merged_away(P, v)) {
      // computed by its GEMM's tiles, or by those of the sibling it is merged into
    } else if (n.op == DAG_OP_GEMM) {
      const bool bf = g.bufs[n.a].dtype == DAG_BF16;
      const int op = bf ? T_GEMM_BF16 : P.tf32w[v] ? T_GEMM_TF32W : P.tf32[v] ? T_GEMM_TF32 : T_GEMM_F32;
      int bm, bn;
      if (bf || P.tf32w[v]) { bm = kBM; bn = P.cfg[v]; }
      else if (P.tf32[v]) { bm = kBM; bn = kTf32BN; }
      else {
        bm = P.cfg[v] == F32_64x64 ? 64 : 128;
        bn = P.cfg[v] == F32_128x128 ? 128 : 64;
      }
      const int M = g.M[v], N = g.N[v];
      const int S = P.nsplit.empty() ? 0 : P.nsplit[v];
      // a split node: every output tile's partials 0..S-2 first, then the
      // finishing partials (so a kernel-by-kernel launch can run them as two grids)
      for (int s = S ? 0 : -1; s < (S ? S : 0); ++s)
        for (int b = 0; b < n.batch; ++b)
          for (int m = 0; m < M; m += bm)
            for (int c = 0; c < N; c += bn) {
              push(op, b * M + m, b * M + std::min(m + bm, M), c, std::min(c + bn, N), P.cfg[v]);
              if (S) P.tiles.back().split = (s << 8) | S;
            }
    } else if (n.op == DAG_OP_SOFTMAX) {
      // memory-bound and latency-bound per SM (a warp keeps eight rows of
      // up to 256 elements in flight).  A softmax that other kernels read:
      // 32..64 rows (16..64 for longer rows), split further while the level
      // has fewer than its share of two tiles per SM, so that its consumers
      // start on early rows.  A softmax nothing reads: one wave of tiles of
      // up to 256 rows, which stream longer per dependency hand-off.
      const bool sink = g.succ[v].empty();
      const double share = (sink ? 1.0 : 2.0) * P.n_sm * ((double)R * C) / std::max(1.0, level_elems[dep[v]]);
      const int lo = C <= 256 ? 32 : 16;
      int rows = sink && C <= 256 ? 256 : C <= 1024 ? 64 : 16;
      if (sink)
        while (rows > lo && (double)((R + rows / 2 - 1) / (rows / 2)) <= share) rows /= 2;
      else
        while (rows > lo && (double)((R + rows - 1) / rows) < share) rows /= 2;
      for (int r = 0; r < R; r += rows) push(T_SOFTMAX, r, std::min(r + rows, R), 0, C, 0);
    } else {
      // at most 64K and at least 4K elements per tile, split further while
      // the level's memory-bound kernels still fit in one tile per SM (their
      // share of the SMs by elements): a tile's fixed cost -- dependency
      // hand-off, one L2 round trip, release -- exceeds its transfer time, so
      // one wave of larger tiles beats two waves of smaller ones
      const double share = 1.0 * P.n_sm * ((double)R * C) / std::max(1.0, level_elems[dep[v]]);
      int rows = 256;
      while (rows > 1 && (long)rows * C > 65536) rows /= 2;
      while (rows > 1 && (double)((R + rows / 2 - 1) / (rows / 2)) <= share && (long)(rows / 2) * C >= 4096)
        rows /= 2;
      for (int r = 0; r < R; r += rows)
        push(n.op == DAG_OP_ADD ? T_ADD : T_UNARY, r, std::min(r + rows, R), 0, C, 0);
    }
    P.node_count[v] = (int)P.tiles.size() - P.node_first[v];
  }
}

// row ranges a tile reads, per input buffer (rows of that buffer)
static int tile_reads(const Graph &g, const TileDesc &t, int buf[3], int r0[3], int r1[3]) {
  const dag_node_desc &n = g.nodes[t.node];
  int k = 0;
  if (n.op == DAG_OP_GEMM) {
    const int M = g.M[t.node], N = g.N[t.node], K = g.K[t.node];
    const int bt = t.r0 / M;
    buf[k] = n.a; r0[k] = t.r0; r1[k] = t.r1; ++k;
    buf[k] = n.b;
    if (n.trans_b) { r0[k] = bt * N + t.c0; r1[k] = bt * N + t.c1; }
    else { r0[k] = bt * K; r1[k] = bt * K + K; }
    ++k;
    if (n.bias >= 0) { buf[k] = n.bias; r0[k] = 0; r1[k] = 1; ++k; }
  } else {
    buf[k] = n.a; r0[k] = t.r0; r1[k] = t.r1; ++k;
    if (n.op == DAG_OP_ADD) { buf[k] = n.b; r0[k] = t.r0; r1[k] = t.r1; ++k; }
  }
  return k;
}

// counters, waits, releases and the tile graph derived from them
static void build_deps(Plan &P, std::vector<std::vector<int>> &tile_pred) {
  Graph &g = P.g;
  const int nt = (int)P.tiles.size();
  // row granularity per written root
  std::vector<int> gran(g.nb, 0), base(g.nb, -1), nblk(g.nb, 0);
  for (int i = 0; i < nt; ++i) {
    const TileDesc &t = P.tiles[i];
    if (split_partial(t)) continue;  // partials write scratch, not the output
    const int root = g.root[tile_out(P, t.node)];
    const int rows = g.bufs[root].rows;
    int gg = gran[root] ? gran[root] : 128;
    while (gg > 16 && ((t.r0 % gg) || ((t.r1 % gg) && t.r1 != rows))) gg /= 2;
    gran[root] = gg;
  }
  int nc = 0;
  for (int r = 0; r < g.nb; ++r)
    if (gran[r]) {
      base[r] = nc;
      nblk[r] = (g.bufs[r].rows + gran[r] - 1) / gran[r];
      nc += nblk[r];
    }
  // split K: one counter per output tile, released by its partials and
  // waited on (S - 1 releases) by the partial that finishes the tile
  std::vector<int> split_ctr(nt, -1);
  {
    std::vector<std::pair<std::pair<int, int64_t>, int>> fin;  // (node, r0 * 2^20 + c0) -> finishing tile
    for (int i = 0; i < nt; ++i)
      if (P.tiles[i].split && !split_partial(P.tiles[i])) {
        split_ctr[i] = nc++;
        fin.push_back({{P.tiles[i].node, (int64_t)P.tiles[i].r0 * (1 << 20) + P.tiles[i].c0}, i});
      }
    std::sort(fin.begin(), fin.end());
    for (int i = 0; i < nt; ++i)
      if (split_partial(P.tiles[i])) {
        const std::pair<int, int64_t> key{P.tiles[i].node, (int64_t)P.tiles[i].r0 * (1 << 20) + P.tiles[i].c0};
        auto it = std::lower_bound(fin.begin(), fin.end(), std::make_pair(key, -1));
        split_ctr[i] = split_ctr[it->second];
      }
  }
  std::vector<uint32_t> target(nc, 0);
  std::vector<std::vector<int>> incr(nc);
  std::vector<std::vector<uint32_t>> rel_of(nt);
  for (int i = 0; i < nt; ++i) {
    const TileDesc &t = P.tiles[i];
    if (split_partial(t)) {
      const int c = split_ctr[i];
      target[c]++;
      incr[c].push_back(i);
      rel_of[i].push_back((uint32_t)c);
      continue;
    }
    const int root = g.root[tile_out(P, t.node)];
    for (int b = t.r0 / gran[root]; b <= (t.r1 - 1) / gran[root]; ++b) {
      const int c = base[root] + b;
      target[c]++;
      incr[c].push_back(i);
      rel_of[i].push_back((uint32_t)c);
    }
  }
  // streamed input flags
  P.flag_of_root.assign(g.nb, -1);
  P.n_flags = 0;
  for (int r = 0; r < g.nb; ++r)
    if (g.bufs[r].view_of < 0 && (g.bufs[r].flags & DAG_BUF_INPUT) && !(g.bufs[r].flags & DAG_BUF_RESIDENT))
      P.flag_of_root[r] = P.n_flags++;
  if (P.opt.debug_never_ready > 0) nc += 1;  // a counter nothing releases
  P.n_counters = nc;

  std::vector<std::vector<Wait>> waits_of(nt);
  tile_pred.assign(nt, {});
  for (int i = 0; i < nt; ++i) {
    const TileDesc &t = P.tiles[i];
    int buf[3], r0[3], r1[3];
    const int k = tile_reads(g, t, buf, r0, r1);
    std::vector<Wait> &W = waits_of[i];
    for (int q = 0; q < k; ++q) {
      const int root = g.root[buf[q]];
      if (P.flag_of_root[root] >= 0) {
        W.push_back(Wait{kWaitFlag | (uint32_t)P.flag_of_root[root], 1u});
        continue;
      }
      if (!gran[root]) continue;  // resident input
      for (int b = r0[q] / gran[root]; b <= (r1[q] - 1) / gran[root]; ++b) {
        const int c = base[root] + b;
        W.push_back(Wait{(uint32_t)c, target[c]});
        for (int u : incr[c]) tile_pred[i].push_back(u);
      }
    }
    if (t.split && !split_partial(t)) {  // the finishing partial waits for the others before its epilogue
      const int c = split_ctr[i];
      W.push_back(Wait{kWaitLate | (uint32_t)c, target[c]});
      for (int u : incr[c]) tile_pred[i].push_back(u);
    }
    int prev = g.nodes[t.node].out;
    if (!split_partial(t))  // fused adds: their other operand's rows, before the epilogue
      for (int e : P.post[t.node]) {
        const dag_node_desc &m = g.nodes[e];
        const int x = m.a == prev ? m.b : m.a;
        prev = m.out;
        if (m.op != DAG_OP_ADD) continue;
        const int root = g.root[x];
        if (P.flag_of_root[root] >= 0) {
          W.push_back(Wait{kWaitFlag | (uint32_t)P.flag_of_root[root], 1u});
          continue;
        }
        if (!gran[root]) continue;  // resident input
        for (int b = t.r0 / gran[root]; b <= (t.r1 - 1) / gran[root]; ++b) {
          const int c = base[root] + b;
          W.push_back(Wait{kWaitLate | (uint32_t)c, target[c]});
          for (int u : incr[c]) tile_pred[i].push_back(u);
        }
      }
    std::sort(W.begin(), W.end(), [](const Wait &a, const Wait &b) { return a.idx < b.idx; });
    W.erase(std::unique(W.begin(), W.end(), [](const Wait &a, const Wait &b) { return a.idx == b.idx; }), W.end());
    std::sort(tile_pred[i].begin(), tile_pred[i].end());
    tile_pred[i].erase(std::unique(tile_pred[i].begin(), tile_pred[i].end()), tile_pred[i].end());
  }
  if (P.opt.debug_never_ready > 0) {
    // the last `debug_never_ready` tiles in creation order wait on a counter no tile releases
    for (int i = std::max(0, nt - P.opt.debug_never_ready); i < nt; ++i)
      waits_of[i].push_back(Wait{(uint32_t)(nc - 1), 1u});
  }
  P.waits.clear();
  P.rels.clear();
  for (int i = 0; i < nt; ++i) {
    TileDesc &t = P.tiles[i];
    t.wait_begin = (int)P.waits.size();
    t.wait_count = (int)waits_of[i].size();
    P.waits.insert(P.waits.end(), waits_of[i].begin(), waits_of[i].end());
    t.rel_begin = (int)P.rels.size();
    t.rel_count = (int)rel_of[i].size();
    P.rels.insert(P.rels.end(), rel_of[i].begin(), rel_of[i].end());
  }
}

// bottom-level ranks and list-scheduled queue order
static void order_tiles(Plan &P, const std::vector<std::vector<int>> &tile_pred) {
  Graph &g = P.g;
  const int nt = (int)P.tiles.size();
  std::vector<double> est(nt);
  for (int i = 0; i < nt; ++i) est[i] = tile_time_us(P, P.tiles[i].node, P.tiles[i]);
  P.node_cost.assign(g.nn, 0.0);
  for (int v = 0; v < g.nn; ++v) {
    if (P.opt.scheduler == DAG_SCHED_RANK_GIVEN && P.opt.node_cost_us) {
      P.node_cost[v] = P.opt.node_cost_us[v];
      continue;
    }
    double t = 0;
    for (int i = P.node_first[v]; i < P.node_first[v] + P.node_count[v]; ++i) t = std::max(t, est[i]);
    const int waves = (P.node_count[v] + P.grid - 1) / P.grid;
    P.node_cost[v] = t * waves;
  }
  P.rank.assign(g.nn, 0.0);
  for (int i = g.nn - 1; i >= 0; --i) {
    const int v = g.topo[i];
    double m = 0;
    for (int w : g.succ[v]) m = std::max(m, P.rank[w]);
    P.rank[v] = P.node_cost[v] + m;
  }
  const bool fifo = P.opt.scheduler == DAG_SCHED_FIFO;
  // the queue's priority: the upward rank, or with DAG_RANK_CRITICAL_PATH the
  // upward plus the downward rank (longest cost path from a root)
  std::vector<double> prio(P.rank);
  if (P.opt.rank_form == DAG_RANK_CRITICAL_PATH) {
    std::vector<double> down(g.nn, 0.0);
    for (int v : g.topo)
      for (int w : g.succ[v]) down[w] = std::max(down[w], down[v] + P.node_cost[v]);
    for (int v = 0; v < g.nn; ++v) prio[v] = P.rank[v] + down[v];
  }

  std::vector<std::vector<int>> tile_succ(nt);
  std::vector<int> indeg(nt, 0);
  for (int i = 0; i < nt; ++i) {
    indeg[i] = (int)tile_pred[i].size();
    for (int u : tile_pred[i]) tile_succ[u].push_back(i);
  }
  std::vector<double> ready_t(nt, 0.0);
  // available set ordered by (rank desc, kernel topo position, creation index)
  auto better = [&](int a, int b) {
    const int va = P.tiles[a].node, vb = P.tiles[b].node;
    if (!fifo && prio[va] != prio[vb]) return prio[va] < prio[vb];
    if (g.topo_pos[va] != g.topo_pos[vb]) return g.topo_pos[va] > g.topo_pos[vb];
    return a > b;
  };
  std::priority_queue<int, std::vector<int>, decltype(better)> avail(better);
  using PI = std::pair<double, int>;
  std::priority_queue<PI, std::vector<PI>, std::greater<PI>> pending;  // by ready time
  std::priority_queue<double, std::vector<double>, std::greater<double>> workers;
  for (int w = 0; w < P.grid; ++w) workers.push(0.0);
  for (int i = 0; i < nt; ++i)
    if (!indeg[i]) pending.push({0.0, i});
  P.queue.clear();
  P.queue_src.clear();
  while (!pending.empty() || !avail.empty()) {
    double now = workers.top();
    if (avail.empty() && pending.top().first > now) now = pending.top().first;
    while (!pending.empty() && pending.top().first <= now) {
      avail.push(pending.top().second);
      pending.pop();
    }
    const int t = avail.top();
    avail.pop();
    // a tile that became available at a later `now` (when no worker was
    // free earlier) still cannot start before its inputs are ready
    const double start = std::max(std::max(now, workers.top()), ready_t[t]);
    workers.pop();
    const double fin = start + est[t];
    workers.push(fin);
    P.queue_src.push_back(t);
    for (int s : tile_succ[t]) {
      ready_t[s] = std::max(ready_t[s], fin);
      if (--indeg[s] == 0) pending.push({ready_t[s], s});
    }
  }
  P.queue.resize(nt);
  for (int q = 0; q < nt; ++q) P.queue[q] = P.tiles[P.queue_src[q]];
}

// algorithmic totals and the critical-path roofline
static void roofline(Plan &P) {
  Graph &g = P.g;
  std::vector<double> cost(g.nn, 0.0);
  P.flops = P.bytes = 0;
  // the DAG's own work: merged siblings count as the kernels they were given as
  const std::vector<dag_node_desc> &nodes = P.orig_nodes.empty() ? g.nodes : P.orig_nodes;
  const std::vector<int> &Ns = P.orig_N.empty() ? g.N : P.orig_N;
  for (int v = 0; v < g.nn; ++v) {
    const dag_node_desc &n = nodes[v];
    double f = 0, b = 0;
    const int in[3] = {n.a, n.b, n.bias};
    const int k = n.op == DAG_OP_GEMM ? (n.bias >= 0 ? 3 : 2) : n.op == DAG_OP_ADD ? 2 : 1;
    for (int q = 0; q < k; ++q) b += (double)g.bufs[in[q]].rows * g.bufs[in[q]].cols * esize(g.bufs[in[q]].dtype);
    b += (double)g.bufs[n.out].rows * g.bufs[n.out].cols * esize(g.bufs[n.out].dtype);
    double peak;
    if (n.op == DAG_OP_GEMM) {
      f = 2.0 * n.batch * (double)g.M[v] * Ns[v] * g.K[v];
      peak = (g.bufs[n.a].dtype == DAG_BF16 ? g_bf16_tflops : P.tf32[v] ? tf32x3_tflops() : g_f32_tflops) * 1e12;
    } else {
      f = (double)g.bufs[n.out].rows * g.bufs[n.out].cols;
      peak = 1e30;  // elementwise work is memory-bound
    }
    P.flops += n.op == DAG_OP_GEMM ? f : 0.0;
    P.bytes += b;
    cost[v] = std::max(n.op == DAG_OP_GEMM ? f / peak : 0.0, b / (g_hbm_gbs * 1e9)) * 1e6;
  }
  std::vector<double> fin(g.nn, 0.0);
  double cp = 0;
  for (int v : g.topo) {
    double s = 0;
    for (int u : g.pred[v]) s = std::max(s, fin[u]);
    fin[v] = s + cost[v];
    cp = std::max(cp, fin[v]);
  }
  P.cp_us = cp;
  double f_bf = 0, f_tc = 0, f_32 = 0;
  for (int v = 0; v < g.nn; ++v)
    if (nodes[v].op == DAG_OP_GEMM) {
      const double f = 2.0 * nodes[v].batch * (double)g.M[v] * Ns[v] * g.K[v];
      const int tv = merged_away(P, v) ? P.merged_into[v] : v;
      (g.bufs[nodes[v].a].dtype == DAG_BF16 ? f_bf : P.tf32[tv] ? f_tc : f_32) += f;
    }
  const double work =
      (f_bf / (g_bf16_tflops * 1e12) + f_tc / (tf32x3_tflops() * 1e12) + f_32 / (g_f32_tflops * 1e12)) * 1e6;
  P.work_us = std::max(cp, std::max(work, P.bytes / (g_hbm_gbs * 1e9) * 1e6));
}

static void plan_tiles(Plan &P) {
  choose_merges(P);   // first: it rewrites the graph the other steps plan
  choose_layouts(P);  // the f32 tile form depends on B's layout
  choose_configs(P);
  choose_fusion(P);
  choose_split(P);
  make_tiles(P);
  std::vector<std::vector<int>> tile_pred;
  build_deps(P, tile_pred);
  if ((int)P.tiles.size() < P.grid) P.grid = std::max(1, (int)P.tiles.size());
  order_tiles(P, tile_pred);
  roofline(P);
}

// Host-only planning (no device): the queue-ordered tiles for a GPU of n_sm SMs
// running one executor CTA per SM.
extern "C" dag_status dag_plan_host(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                                    const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts, int n_sm,
                                    int32_t *out6, int cap, int *n_tiles, dag_plan_info *info) {
  if (!n_tiles || n_sm <= 0) return fail(DAG_EINVAL, "null n_tiles or n_sm <= 0");
  Plan P;
  if (opts) P.opt = *opts;
  dag_status s = build_graph(nodes, n_nodes, edges, n_edges, buffers, n_buffers, P.g);
  if (s) return s;
  P.n_sm = n_sm;
  P.grid = P.opt.max_ctas > 0 ? std::min(n_sm, P.opt.max_ctas) : n_sm;
  plan_tiles(P);
  const int nt = (int)P.queue.size();
  *n_tiles = nt;
  for (int i = 0; out6 && i < nt && i < cap; ++i) {
    const TileDesc &t = P.queue[i];
    const int32_t r[6] = {t.node, t.r0, t.r1, t.c0, t.c1, t.cfg | (t.split << 16)};
    memcpy(out6 + 6 * i, r, sizeof r);
  }
  if (info) {
    info->n_tiles = nt;
    info->n_counters = P.n_counters;
    info->n_waits = (int)P.waits.size();
    info->grid = P.grid;
    info->smem_bytes = 0;
    info->flops = P.flops;
    info->bytes = P.bytes;
    info->critical_path_us = P.cp_us;
    info->work_bound_us = P.work_us;
  }
  return DAG_OK;
}

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct dag_handle {
  Plan P;
  int device = 0;
  // device memory
  void *arena = nullptr;      // buffers
  size_t arena_bytes = 0;
  void *meta = nullptr;       // plan arrays
  float *split_scratch = nullptr;  // split K partial sums
  void *staging = nullptr;         // upload area of weights kept transposed
  cudaEvent_t ev_staging = nullptr;
  bool staging_used = false;
  std::vector<char *> dptr;   // per buffer (view-adjusted)
  std::vector<int64_t> ld;    // per buffer row pitch (elements)
  ExecParams xp{};            // persistent-mode parameters
  TileDesc *d_coarse = nullptr;
  TraceRec *d_trace = nullptr;
  uint32_t *d_flags = nullptr;
  Ctrl *d_ctrl = nullptr;
  // host side
  std::vector<const void *> host_in;
  std::vector<void *> host_out;
  std::vector<char> resident_dirty;
  cudaStream_t up[2] = {nullptr, nullptr}, down = nullptr;
  cudaEvent_t ev_done = nullptr, ev_read = nullptr;
  uint32_t epoch = 0;
  bool in_flight = false, reading = false;
  dag_status poisoned = DAG_OK;
  int last_mode = 0;
  // CUDA graph of the persistent launch (use_graph)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  double tuned_us = 0.0;
  // command-queue executor (dag_submit_cq): streams and per-kernel / per-buffer events
  std::vector<cudaStream_t> cq_q;
  std::vector<cudaEvent_t> cq_beg, cq_end, cq_buf;
  cudaEvent_t cq_t0 = nullptr;
};

static void free_handle(dag_handle *h) {
  if (!h) return;
  for (cudaStream_t q : h->cq_q) cudaStreamDestroy(q);
  for (auto *v : {&h->cq_beg, &h->cq_end, &h->cq_buf})
    for (cudaEvent_t e : *v)
      if (e) cudaEventDestroy(e);
  if (h->cq_t0) cudaEventDestroy(h->cq_t0);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->arena) cudaFree(h->arena);
  if (h->meta) cudaFree(h->meta);
  if (h->split_scratch) cudaFree(h->split_scratch);
  if (h->staging) cudaFree(h->staging);
  if (h->ev_staging) cudaEventDestroy(h->ev_staging);
  for (auto &s : h->up)
    if (s) cudaStreamDestroy(s);
  if (h->down) cudaStreamDestroy(h->down);
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->ev_read) cudaEventDestroy(h->ev_read);
  delete h;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static dag_status encode_map(CUtensorMap *m, const void *base, uint64_t d0, uint64_t d1, uint64_t d2,
                             uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t b0, uint32_t b1,
                             int dtype = DAG_BF16, CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B) {
  const cuuint64_t dims[3] = {d0, d1, d2};
  const cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
  const cuuint32_t box[3] = {b0, b1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = p_encode_tiled(m, dtype == DAG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              3, const_cast<void *>(base), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(DAG_EUNSUPPORTED, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return DAG_OK;
}

// Output map of the TMA-store epilogue: dims {N, M, batch}, box {128 bytes of
// columns, 32 rows, 1}, 128-byte swizzle (the layout the epilogue stages).
static dag_status encode_out_map(CUtensorMap *m, const void *base, int dtype, uint64_t N, uint64_t M, uint64_t B,
                                 uint64_t ld_elems) {
  const int es = esize(dtype);
  const cuuint64_t dims[3] = {N, M, B};
  const cuuint64_t strides[2] = {ld_elems * es, M * ld_elems * es};
  const cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)kEpiRows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = p_encode_tiled(m, dtype == DAG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              3, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(DAG_EUNSUPPORTED, "cuTensorMapEncodeTiled (output) failed (%d)", (int)r);
  return DAG_OK;
}

// Tensor maps of a tensor-core GEMM node (bf16, or f32 split into tf32):
// A box {K block, 128 rows}; B K-major box {K block, BN}, MN-major boxes of
// 128 bytes of columns x K block; all with the 128-byte swizzle.  Plus the
// output map of the TMA-store epilogue when C is 16-byte aligned.
static dag_status gemm_maps(const Plan &P, int v, NodeParams &q, std::vector<CUtensorMap> &maps) {
  const dag_node_desc &n = P.g.nodes[v];
  if (n.op != DAG_OP_GEMM || (q.a_dt != DAG_BF16 && !P.tf32[v])) return DAG_OK;
  if (((uintptr_t)q.A % 16) || ((uintptr_t)q.B % 16))
    return fail(DAG_EUNSUPPORTED, "node %d: tensor-core GEMM operand view not 16-byte aligned", v);
  const int M = q.M, N = q.N, K = q.K, B = n.batch;
  const int dt = q.a_dt, es = esize(dt);
  const uint32_t kb = dt == DAG_BF16 ? kBK : kBKF;          // 128 bytes of K
  const uint32_t bn = dt == DAG_BF16 ? P.cfg[v] : kTf32BN;
  CUtensorMap ma, mb;
  dag_status s;
  if (P.tf32w[v]) {
    // the wide f32 form: boxes {16 (K), 128} and {16 (K), BN}, 64-byte swizzle, B K-major
    if (!q.trans_b) return fail(DAG_EUNSUPPORTED, "node %d: wide f32 tiles need B K-major", v);
    const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_64B;
    if ((s = encode_map(&ma, q.A, K, M, B, q.lda * es, (uint64_t)M * q.lda * es, kBKW, kBM, dt, sw))) return s;
    if ((s = encode_map(&mb, q.B, K, N, B, q.ldb * es, (uint64_t)N * q.ldb * es, kBKW, P.cfg[v], dt, sw))) return s;
  } else {
    if ((s = encode_map(&ma, q.A, K, M, B, q.lda * es, (uint64_t)M * q.lda * es, kb, kBM, dt))) return s;
    if (q.trans_b) s = encode_map(&mb, q.B, K, N, B, q.ldb * es, (uint64_t)N * q.ldb * es, kb, bn, dt);
    else s = encode_map(&mb, q.B, N, K, B, q.ldb * es, (uint64_t)K * q.ldb * es, 128 / es, kb, dt);
    if (s) return s;
  }
  q.tmap_a = (int)maps.size(); maps.push_back(ma);
  q.tmap_b = (int)maps.size(); maps.push_back(mb);
  q.tmap_c = -1;
  if ((uintptr_t)q.C % 16 == 0) {
    CUtensorMap mc;
    if ((s = encode_out_map(&mc, q.C, q.c_dt, N, M, B, q.ldc))) return s;
    q.tmap_c = (int)maps.size(); maps.push_back(mc);
  }
  return DAG_OK;
}

// Kernel parameters of node v over the view-adjusted device buffers dptr /
// ld, the elementwise kernels fused into its epilogue, and its tensor maps.
static dag_status fill_params(const Plan &P, int v, char *const *dptr, const int64_t *ld, NodeParams &q,
                              std::vector<CUtensorMap> &maps) {
  const Graph &g = P.g;
  const dag_node_desc &n = g.nodes[v];
  memset(&q, 0, sizeof q);
  if (merged_away(P, v)) {  // no tiles: the merged sibling computes it
    q.tmap_a = q.tmap_b = q.tmap_c = -1;
    return DAG_OK;
  }
  q.A = dptr[n.a];
  q.lda = ld[n.a];
  q.a_dt = g.bufs[n.a].dtype;
  if (n.op == DAG_OP_GEMM || n.op == DAG_OP_ADD) { q.B = dptr[n.b]; q.ldb = ld[n.b]; q.b_dt = g.bufs[n.b].dtype; }
  if (n.op == DAG_OP_GEMM && n.bias >= 0) { q.bias = dptr[n.bias]; q.bias_dt = g.bufs[n.bias].dtype; }
  const int out = tile_out(P, v);
  q.C = dptr[out];
  q.ldc = ld[out];
  q.c_dt = g.bufs[out].dtype;
  q.o_dt = g.bufs[n.out].dtype;
  q.M = g.M[v]; q.N = g.N[v]; q.K = g.K[v]; q.batch = n.op == DAG_OP_GEMM ? n.batch : 1;
  // a weight kept transposed is read K-major
  q.trans_b = n.trans_b || (n.op == DAG_OP_GEMM && P.store_t[g.root[n.b]]);
  q.act = n.act; q.scale = n.scale;
  q.tmap_a = q.tmap_b = q.tmap_c = -1;
  // 16-byte vector paths: every operand starts on a 16-byte boundary (row
  // pitches are multiples of 16 bytes)
  bool vec = true;
  int in[3];
  const int k = g.inputs(v, in);
  for (int i = 0; i < k; ++i) vec &= ((uintptr_t)dptr[in[i]] % 16) == 0;
  vec &= ((uintptr_t)dptr[out] % 16) == 0;
  q.vec = vec ? 1 : 0;
  int prev = n.out;
  for (int e : P.post[v]) {
    const dag_node_desc &m = g.nodes[e];
    PostOp &o = q.post[q.n_post++];
    o.act = m.act;
    o.out_dt = g.bufs[m.out].dtype;
    if (m.op == DAG_OP_ADD) {
      const int x = m.a == prev ? m.b : m.a;
      o.X = dptr[x];
      o.ldx = ld[x];
      o.x_dt = g.bufs[x].dtype;
      o.xvec = ((uintptr_t)dptr[x] % 16) == 0 && (ld[x] * esize(o.x_dt)) % 16 == 0;
    }
    prev = m.out;
  }
  return gemm_maps(P, v, q, maps);
}

static dag_status create_impl(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                              const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts,
                              dag_handle **out) {
  if (!out) return fail(DAG_EINVAL, "null output handle");
  *out = nullptr;
  dag_status s = init_driver();
  if (s) return s;
  dag_handle *h = new (std::nothrow) dag_handle();
  if (!h) return fail(DAG_ENOMEM, "host allocation");
  Plan &P = h->P;
  if (opts) P.opt = *opts;
  if (!P.opt.timeout_ns) P.opt.timeout_ns = 2000000000ull;
  if ((s = build_graph(nodes, n_nodes, edges, n_edges, buffers, n_buffers, P.g))) { free_handle(h); return s; }
  Graph &g = P.g;
  if (cudaGetDevice(&h->device) != cudaSuccess) { free_handle(h); return fail(DAG_EDEVICE, "no CUDA device"); }
  cudaDeviceGetAttribute(&P.n_sm, cudaDevAttrMultiProcessorCount, h->device);
  const int per_sm = std::max(1, max_coresident_ctas_per_sm());
  P.grid = P.n_sm * per_sm;
  if (P.opt.max_ctas > 0) P.grid = std::min(P.grid, P.opt.max_ctas);

  plan_tiles(P);

  // ---- device buffers: one arena, row pitch a multiple of 16 elements ----
  h->dptr.assign(g.nb, nullptr);
  h->ld.assign(g.nb, 0);
  std::vector<size_t> off(g.nb, 0);
  size_t total = 0;
  size_t stage_bytes = 0;
  for (int b = 0; b < g.nb; ++b) {
    if (g.bufs[b].view_of >= 0) continue;
    const int es = esize(g.bufs[b].dtype);
    // a weight kept transposed: batch blocks of N x K
    const int64_t rows = P.store_t[b] ? (int64_t)P.t_batch[b] * P.t_N[b] : g.bufs[b].rows;
    h->ld[b] = round_up(P.store_t[b] ? P.t_K[b] : g.bufs[b].cols, 16);
    off[b] = total;
    total = align_up(total + (size_t)rows * h->ld[b] * es, 1024);
    if (P.store_t[b]) stage_bytes = std::max(stage_bytes, (size_t)g.bufs[b].rows * g.bufs[b].cols * es);
  }
  if (stage_bytes && (cudaMalloc(&h->staging, stage_bytes) != cudaSuccess ||
                      cudaEventCreateWithFlags(&h->ev_staging, cudaEventDisableTiming) != cudaSuccess)) {
    free_handle(h);
    return fail(DAG_ENOMEM, "weight staging (%zu bytes)", stage_bytes);
  }
  if (total && cudaMalloc(&h->arena, total) != cudaSuccess) { free_handle(h); return fail(DAG_ENOMEM, "device buffers (%zu bytes)", total); }
  h->arena_bytes = total;
  if (total) cudaMemset(h->arena, 0, total);
  for (int b = 0; b < g.nb; ++b) {
    const int r = g.root[b];
    h->ld[b] = h->ld[r];
    h->dptr[b] = (char *)h->arena + off[r] + (size_t)g.coff[b] * esize(g.bufs[b].dtype);
  }

  // ---- node parameters and tensor maps ----
  const int nn = g.nn, nt = (int)P.tiles.size();
  std::vector<NodeParams> np(std::max(1, nn));
  std::vector<CUtensorMap> maps;
  for (int v = 0; v < nn; ++v)
    if ((s = fill_params(P, v, h->dptr.data(), h->ld.data(), np[v], maps))) { free_handle(h); return s; }
  // split K scratch: (S - 1) blocks of 128 x BN f32 per output tile
  {
    std::vector<size_t> soff(nn, 0);
    size_t stotal = 0;
    for (int v = 0; v < nn; ++v)
      if (P.nsplit[v] >= 2) {
        soff[v] = stotal;
        const int bn = P.cfg[v];
        const size_t tiles = (size_t)g.nodes[v].batch * ((g.M[v] + kBM - 1) / kBM) * ((g.N[v] + bn - 1) / bn);
        stotal += (size_t)(P.nsplit[v] - 1) * tiles * kBM * bn;
      }
    if (stotal) {
      if (cudaMalloc(&h->split_scratch, stotal * sizeof(float)) != cudaSuccess) {
        free_handle(h);
        return fail(DAG_ENOMEM, "split-K scratch (%zu bytes)", stotal * sizeof(float));
      }
      for (int v = 0; v < nn; ++v)
        if (P.nsplit[v] >= 2) np[v].scratch = h->split_scratch + soff[v];
    }
  }

  // ---- plan arrays in one device block ----
  std::vector<TileDesc> coarse(P.tiles);
  size_t o_maps = 0;
  size_t o_tiles = align_up(o_maps + maps.size() * sizeof(CUtensorMap), 256);
  size_t o_coarse = align_up(o_tiles + (size_t)nt * sizeof(TileDesc), 256);
  size_t o_waits = align_up(o_coarse + (size_t)nt * sizeof(TileDesc), 256);
  size_t o_rels = align_up(o_waits + P.waits.size() * sizeof(Wait), 256);
  size_t o_nodes = align_up(o_rels + P.rels.size() * sizeof(uint32_t), 256);
  size_t o_cnt = align_up(o_nodes + np.size() * sizeof(NodeParams), 256);
  size_t o_flags = align_up(o_cnt + (size_t)std::max(1, P.n_counters) * 4, 256);
  size_t o_ctrl = align_up(o_flags + (size_t)std::max(1, P.n_flags) * 4, 256);
  size_t o_trace = align_up(o_ctrl + sizeof(Ctrl), 256);
  size_t mtotal = align_up(o_trace + (size_t)std::max(1, nt) * sizeof(TraceRec), 256);
  if (cudaMalloc(&h->meta, mtotal) != cudaSuccess) { free_handle(h); return fail(DAG_ENOMEM, "plan arrays"); }
  char *m = (char *)h->meta;
  cudaMemset(m, 0, mtotal);
  auto put = [&](size_t o, const void *src, size_t n) { return n ? cudaMemcpy(m + o, src, n, cudaMemcpyHostToDevice) : cudaSuccess; };
  if (put(o_maps, maps.data(), maps.size() * sizeof(CUtensorMap)) || put(o_tiles, P.queue.data(), (size_t)nt * sizeof(TileDesc)) ||
      put(o_coarse, coarse.data(), (size_t)nt * sizeof(TileDesc)) || put(o_waits, P.waits.data(), P.waits.size() * sizeof(Wait)) ||
      put(o_rels, P.rels.data(), P.rels.size() * sizeof(uint32_t)) || put(o_nodes, np.data(), np.size() * sizeof(NodeParams))) {
    free_handle(h);
    return fail(DAG_EDEVICE, "plan upload: %s", cudaGetErrorString(cudaGetLastError()));
  }
  ExecParams &x = h->xp;
  x.tiles = (const TileDesc *)(m + o_tiles);
  x.n_tiles = nt;
  x.mode = 0;
  x.tile_begin = 0;
  x.trace_on = P.opt.trace ? 1 : 0;
  x.fused = std::any_of(P.post.begin(), P.post.end(), [](const std::vector<int> &c) { return !c.empty(); }) ? 1 : 0;
  x.waits = (const Wait *)(m + o_waits);
  x.rels = (const uint32_t *)(m + o_rels);
  x.nodes = (const NodeParams *)(m + o_nodes);
  x.tmaps = (const CUtensorMap *)(m + o_maps);
  x.counters = (uint32_t *)(m + o_cnt);
  x.flags = (uint32_t *)(m + o_flags);
  x.ctrl = (Ctrl *)(m + o_ctrl);
  x.trace = (TraceRec *)(m + o_trace);
  x.timeout_ns = P.opt.timeout_ns;
  h->d_coarse = (TileDesc *)(m + o_coarse);
  h->d_flags = x.flags;
  h->d_ctrl = x.ctrl;
  h->d_trace = x.trace;

  h->host_in.assign(g.nb, nullptr);
  h->host_out.assign(g.nb, nullptr);
  h->resident_dirty.assign(g.nb, 0);
  for (auto &st : h->up)
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { free_handle(h); return fail(DAG_EDEVICE, "stream"); }
  if (cudaStreamCreateWithFlags(&h->down, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_read, cudaEventDisableTiming) != cudaSuccess) {
    free_handle(h);
    return fail(DAG_EDEVICE, "stream/event creation");
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { free_handle(h); return fail(DAG_EDEVICE, "setup: %s", cudaGetErrorString(cudaGetLastError())); }
  *out = h;
  return DAG_OK;
}

// Median device time (us) of `runs` fine-grained submissions of h on `st`.
static dag_status time_handle(dag_handle *h, cudaStream_t st, int runs, double *us);

// The autotuner: plans with each tile policy (the concurrency heuristic, or
// every bf16 GEMM at BN = 256 / 128) and each queue order (ranked, FIFO) are
// built and timed on the device (zeroed buffers, one warm-up, median of three
// runs); the fastest is kept.  The shape search is empirical: whatever the
// time model says, the measured plan wins.
extern "C" dag_status dag_create(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                                 const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts,
                                 dag_handle **out) {
  if (!opts || !opts->autotune) return create_impl(nodes, n_nodes, edges, n_edges, buffers, n_buffers, opts, out);
  dag_options best = *opts, cand = *opts;
  best.autotune = cand.autotune = 0;
  cand.trace = 0;
  cand.use_graph = 0;
  double best_us = 1e300;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(DAG_EDEVICE, "stream");
  const int tiles[3] = {0, 256, 128};
  const int scheds[2] = {DAG_SCHED_RANK_MODEL, DAG_SCHED_FIFO};
  for (int ti = 0; ti < 3; ++ti)
    for (int si = 0; si < 2; ++si) {
      cand.tile_override = tiles[ti];
      cand.scheduler = scheds[si];
      if (opts->scheduler == DAG_SCHED_RANK_GIVEN && si == 0) cand.scheduler = DAG_SCHED_RANK_GIVEN;
      dag_handle *h = nullptr;
      dag_status s = create_impl(nodes, n_nodes, edges, n_edges, buffers, n_buffers, &cand, &h);
      if (s) { cudaStreamDestroy(st); return s; }
      double us = 0;
      s = time_handle(h, st, 3, &us);
      free_handle(h);
      if (s) { cudaStreamDestroy(st); return s; }
      if (us < best_us) {
        best_us = us;
        best.tile_override = cand.tile_override;
        best.scheduler = cand.scheduler;
      }
    }
  cudaStreamDestroy(st);
  dag_status s = create_impl(nodes, n_nodes, edges, n_edges, buffers, n_buffers, &best, out);
  if (!s) (*out)->tuned_us = best_us;
  return s;
}

extern "C" dag_status dag_batch_create(const dag_batch_item *items, int n_items, const dag_options *opts,
                                       dag_handle **out) {
  if (!out || n_items < 0 || (n_items && !items)) return fail(DAG_EINVAL, "bad batch arguments");
  std::vector<dag_node_desc> nodes;
  std::vector<dag_buffer_desc> bufs;
  for (int i = 0; i < n_items; ++i) {
    const dag_batch_item &it = items[i];
    if (it.n_nodes < 0 || it.n_buffers < 0 || (it.n_nodes && !it.nodes) || (it.n_buffers && !it.buffers))
      return fail(DAG_EINVAL, "batch item %d: bad arrays", i);
    const int boff = (int)bufs.size();
    for (int b = 0; b < it.n_buffers; ++b) {
      dag_buffer_desc d = it.buffers[b];
      if (d.view_of >= 0) {
        if (d.view_of >= it.n_buffers) return fail(DAG_EINVAL, "batch item %d buffer %d: bad view parent", i, b);
        d.view_of += boff;
      }
      bufs.push_back(d);
    }
    for (int v = 0; v < it.n_nodes; ++v) {
      dag_node_desc n = it.nodes[v];
      auto remap = [&](int32_t &id) -> bool {
        if (id < 0) return true;
        if (id >= it.n_buffers) return false;
        id += boff;
        return true;
      };
      if (!remap(n.a) || !remap(n.b) || !remap(n.bias) || !remap(n.out))
        return fail(DAG_EINVAL, "batch item %d node %d: buffer id out of range", i, v);
      nodes.push_back(n);
    }
  }
  return dag_create(nodes.data(), (int)nodes.size(), nullptr, 0, bufs.data(), (int)bufs.size(), opts, out);
}

static dag_status check_handle(dag_handle *h) {
  if (!h) return fail(DAG_EINVAL, "null handle");
  if (h->poisoned) return fail(h->poisoned, "handle poisoned by an earlier device error");
  return DAG_OK;
}

extern "C" dag_status dag_set_input(dag_handle *h, int buf, const void *host_ptr) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (!caller_buf(h->P, buf) || !(h->P.g.bufs[buf].flags & DAG_BUF_INPUT))
    return fail(DAG_EINVAL, "buffer %d is not an input", buf);
  if (h->in_flight) return fail(DAG_EBUSY, "a submit is in flight");
  h->host_in[buf] = host_ptr;
  if (h->P.g.bufs[buf].flags & DAG_BUF_RESIDENT) h->resident_dirty[buf] = host_ptr ? 1 : 0;
  return DAG_OK;
}

extern "C" dag_status dag_set_output(dag_handle *h, int buf, void *host_ptr) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (!caller_buf(h->P, buf)) return fail(DAG_EINVAL, "bad buffer %d", buf);
  if (h->P.store_t[h->P.g.root[buf]])
    return fail(DAG_EINVAL, "buffer %d is a weight kept transposed on the device: read it with dag_get_output", buf);
  if (h->in_flight) return fail(DAG_EBUSY, "a submit is in flight");
  h->host_out[buf] = host_ptr;
  return DAG_OK;
}

static cudaError_t copy_h2d(dag_handle *h, int b, cudaStream_t st) {
  const dag_buffer_desc &d = h->P.g.bufs[b];
  const Plan &P = h->P;
  const int r = P.g.root[b];
  if (r != b && P.store_t[r]) {
    // a merged sibling's weight (K x N, batch 1): its slice of the parent kept
    // transposed is rows [coff, coff + N) of the parent's N x K form
    cudaError_t e = cudaSuccess;
    if (h->staging_used) e = cudaStreamWaitEvent(st, h->ev_staging, 0);
    if (!e) e = cudaMemcpyAsync(h->staging, h->host_in[b], (size_t)d.rows * d.cols * esize(d.dtype),
                                cudaMemcpyHostToDevice, st);
    char *dst = h->dptr[r] + (size_t)P.g.coff[b] * h->ld[r] * esize(d.dtype);
    if (!e) e = launch_transpose(h->staging, d.cols, dst, h->ld[r], 1, d.rows, d.cols, esize(d.dtype), st);
    if (!e) e = cudaEventRecord(h->ev_staging, st);
    h->staging_used = true;
    return e;
  }
  if (P.store_t[b]) {  // through the staging area (one upload at a time, in any stream), then transposed
    cudaError_t e = cudaSuccess;
    if (h->staging_used) e = cudaStreamWaitEvent(st, h->ev_staging, 0);
    if (!e) e = cudaMemcpyAsync(h->staging, h->host_in[b], (size_t)d.rows * d.cols * esize(d.dtype),
                                cudaMemcpyHostToDevice, st);
    if (!e) e = launch_transpose(h->staging, d.cols, h->dptr[b], h->ld[b], P.t_batch[b], P.t_K[b], P.t_N[b],
                                 esize(d.dtype), st);
    if (!e) e = cudaEventRecord(h->ev_staging, st);
    h->staging_used = true;
    return e;
  }
  const size_t w = (size_t)d.cols * esize(d.dtype);
  if (h->ld[b] == d.cols)  // rows back to back on both sides: one linear copy
    return cudaMemcpyAsync(h->dptr[b], h->host_in[b], w * d.rows, cudaMemcpyHostToDevice, st);
  return cudaMemcpy2DAsync(h->dptr[b], (size_t)h->ld[b] * esize(d.dtype), h->host_in[b], w, w, d.rows,
                           cudaMemcpyHostToDevice, st);
}

static dag_status enqueue_readbacks(dag_handle *h, cudaStream_t stream) {
  h->reading = false;
  for (int b = 0; b < h->P.g.nb; ++b) {
    if (!h->host_out[b]) continue;
    if (!h->reading) {
      CUDA_TRY(cudaStreamWaitEvent(h->down, h->ev_done, 0));
      h->reading = true;
    }
    const dag_buffer_desc &d = h->P.g.bufs[b];
    const size_t w = (size_t)d.cols * esize(d.dtype);
    if (h->ld[b] == d.cols)  // rows back to back on both sides: one linear copy
      CUDA_TRY(cudaMemcpyAsync(h->host_out[b], h->dptr[b], w * d.rows, cudaMemcpyDeviceToHost, h->down));
    else
      CUDA_TRY(cudaMemcpy2DAsync(h->host_out[b], w, h->dptr[b], (size_t)h->ld[b] * esize(d.dtype), w, d.rows,
                                 cudaMemcpyDeviceToHost, h->down));
  }
  if (h->reading) CUDA_TRY(cudaEventRecord(h->ev_read, h->down));
  (void)stream;
  return DAG_OK;
}

extern "C" dag_status dag_submit(dag_handle *h, void *stream_) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (h->in_flight) return fail(DAG_EBUSY, "previous submit not waited for");
  cudaStream_t stream = (cudaStream_t)stream_;
  Plan &P = h->P;
  // resident inputs that changed: uploaded in stream order before the launch
  for (int b = 0; b < P.g.nb; ++b)
    if (h->resident_dirty[b]) {
      CUDA_TRY(copy_h2d(h, b, stream));
      h->resident_dirty[b] = 0;
    }
  // streamed inputs: copy on an upload stream, then raise the ready flag;
  // tiles that read the buffer acquire the flag (the copy engine overlaps compute)
  const uint32_t want = h->epoch + 1;
  int k = 0;
  for (int b = 0; b < P.g.nb; ++b) {
    const int f = P.flag_of_root[b];
    if (f < 0) continue;
    CUdeviceptr flag = (CUdeviceptr)(h->d_flags + f);
    if (h->host_in[b]) {
      cudaStream_t st = h->up[k++ & 1];
      CUDA_TRY(copy_h2d(h, b, st));
      if (p_write_value32((CUstream)st, flag, want, CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS)
        return fail(DAG_EDEVICE, "cuStreamWriteValue32");
    } else if (p_write_value32((CUstream)stream, flag, want, CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS) {
      return fail(DAG_EDEVICE, "cuStreamWriteValue32");
    }
  }
  if (P.opt.trace && P.tiles.size()) {
    CUDA_TRY(cudaMemsetAsync(h->d_trace, 0, P.tiles.size() * sizeof(TraceRec), stream));
    CUDA_TRY(cudaMemsetAsync(&h->d_ctrl->t_enter, 0xFF, sizeof(uint64_t), stream));  // the launch's window
    CUDA_TRY(cudaMemsetAsync(&h->d_ctrl->t_exit, 0, sizeof(uint64_t), stream));
  }
  if (P.tiles.size() && P.opt.use_graph) {
    if (!h->gexec) {  // capture the persistent launch once; replays reuse it
      if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t le = launch_persistent(h->xp, P.grid, h->cap_stream);
      const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &h->graph);
      if (le != cudaSuccess || ce != cudaSuccess) return fail(DAG_EDEVICE, "graph capture failed");
      CUDA_TRY(cudaGraphInstantiate(&h->gexec, h->graph, 0));
    }
    CUDA_TRY(cudaGraphLaunch(h->gexec, stream));
  } else if (P.tiles.size()) {
    CUDA_TRY(launch_persistent(h->xp, P.grid, stream));
  }
  CUDA_TRY(cudaEventRecord(h->ev_done, stream));
  if ((s = enqueue_readbacks(h, stream))) return s;
  h->epoch++;
  h->in_flight = true;
  h->last_mode = 0;
  return DAG_OK;
}

// One kernel's tiles as coarse grids (no waits inside a grid): a split node
// runs its partials first and its finishing tiles in a second grid.
static cudaError_t launch_node_coarse(const ExecParams &x, const Plan &P, int v, cudaStream_t st) {
  const int first = P.node_first[v], count = P.node_count[v];
  if (!count) return cudaSuccess;
  int partials = 0;
  while (partials < count && split_partial(P.tiles[first + partials])) ++partials;
  cudaError_t e = cudaSuccess;
  if (partials) e = launch_coarse(x, first, partials, st);
  if (!e && count > partials) e = launch_coarse(x, first + partials, count - partials, st);
  return e;
}

// The kernel whose tiles launch in kernel v's turn of a kernel-by-kernel
// order (-1: none): a GEMM with fused kernels launches in the last one's turn,
// when every operand of the chain has been produced.
static int launch_in_turn(const Plan &P, int v) {
  const int head = P.absorbed_by[v];
  if (head >= 0) return P.post[head].back() == v ? head : -1;
  return P.post[v].empty() ? v : -1;
}

extern "C" dag_status dag_submit_coarse(dag_handle *h, void *stream_) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (h->in_flight) return fail(DAG_EBUSY, "previous submit not waited for");
  cudaStream_t stream = (cudaStream_t)stream_;
  Plan &P = h->P;
  for (int b = 0; b < P.g.nb; ++b) {
    if (h->resident_dirty[b]) { CUDA_TRY(copy_h2d(h, b, stream)); h->resident_dirty[b] = 0; }
    else if (P.flag_of_root[b] >= 0 && h->host_in[b]) CUDA_TRY(copy_h2d(h, b, stream));
  }
  ExecParams x = h->xp;
  x.tiles = h->d_coarse;
  if (P.opt.trace && P.tiles.size()) {
    CUDA_TRY(cudaMemsetAsync(h->d_trace, 0, P.tiles.size() * sizeof(TraceRec), stream));
    CUDA_TRY(cudaMemsetAsync(&h->d_ctrl->t_enter, 0xFF, sizeof(uint64_t), stream));  // the launch's window
    CUDA_TRY(cudaMemsetAsync(&h->d_ctrl->t_exit, 0, sizeof(uint64_t), stream));
  }
  for (int v : P.g.topo)
    if (launch_in_turn(P, v) >= 0) CUDA_TRY(launch_node_coarse(x, P, launch_in_turn(P, v), stream));
  CUDA_TRY(cudaEventRecord(h->ev_done, stream));
  if ((s = enqueue_readbacks(h, stream))) return s;
  h->in_flight = true;
  h->last_mode = 1;
  return DAG_OK;
}

static dag_status poll_event(cudaEvent_t ev, uint64_t timeout_ns) {
  const auto t0 = std::chrono::steady_clock::now();
  for (uint64_t n = 0;; ++n) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return DAG_OK;
    if (e != cudaErrorNotReady) return fail(DAG_EDEVICE, "device error: %s", cudaGetErrorString(e));
    if ((uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0).count() > timeout_ns)
      return fail(DAG_ETIMEOUT, "dag_wait timed out");
    if (n > 2000) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

extern "C" dag_status dag_wait(dag_handle *h, uint64_t timeout_ns) {
  if (!h) return fail(DAG_EINVAL, "null handle");
  if (h->poisoned) return fail(h->poisoned, "handle poisoned by an earlier device error");
  if (!h->in_flight) return DAG_OK;
  dag_status s = poll_event(h->reading ? h->ev_read : h->ev_done, timeout_ns ? timeout_ns : ~0ull);
  if (s == DAG_ETIMEOUT) return s;
  h->in_flight = false;
  if (s) { h->poisoned = s; return s; }
  Ctrl c;
  if (cudaMemcpy(&c, h->d_ctrl, sizeof c, cudaMemcpyDeviceToHost) != cudaSuccess) {
    h->poisoned = DAG_EDEVICE;
    return fail(DAG_EDEVICE, "reading the device error word");
  }
  if (c.err_code) {
    h->poisoned = c.err_code == E_DEP_TIMEOUT || c.err_code == E_PIPE_TIMEOUT ? DAG_ETIMEOUT : DAG_EDEVICE;
    return fail(h->poisoned, "device error %u at tile %u", c.err_code, c.err_tile);
  }
  return DAG_OK;
}

static dag_status time_handle(dag_handle *h, cudaStream_t st, int runs, double *us) {
  cudaEvent_t a, b;
  CUDA_TRY(cudaEventCreate(&a));
  CUDA_TRY(cudaEventCreate(&b));
  std::vector<float> ms;
  dag_status s = DAG_OK;
  for (int r = 0; r <= runs && !s; ++r) {
    cudaEventRecord(a, st);
    if ((s = dag_submit(h, st))) break;
    cudaEventRecord(b, st);
    if ((s = dag_wait(h, 60ull * 1000000000ull))) break;
    float t = 0;
    cudaEventElapsedTime(&t, a, b);
    if (r) ms.push_back(t);  // the first run warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s) return s;
  std::sort(ms.begin(), ms.end());
  *us = ms.empty() ? 0.0 : ms[ms.size() / 2] * 1e3;
  return DAG_OK;
}

extern "C" dag_status dag_poll(dag_handle *h) {
  if (!h) return fail(DAG_EINVAL, "null handle");
  if (h->poisoned) return fail(h->poisoned, "handle poisoned by an earlier device error");
  if (!h->in_flight) return DAG_OK;
  const cudaError_t e = cudaEventQuery(h->reading ? h->ev_read : h->ev_done);
  if (e == cudaErrorNotReady) return DAG_EBUSY;
  return dag_wait(h, 0);
}

extern "C" dag_status dag_get_output(dag_handle *h, int buf, void *host_ptr) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (!caller_buf(h->P, buf) || !host_ptr) return fail(DAG_EINVAL, "bad buffer or pointer");
  if (h->in_flight) return fail(DAG_EBUSY, "call dag_wait first");
  const dag_buffer_desc &d = h->P.g.bufs[buf];
  const int es = esize(d.dtype);
  const size_t w = (size_t)d.cols * es;
  const Plan &P = h->P;
  const int root = P.g.root[buf];
  if (root != buf && P.store_t[root]) {  // a merged sibling's weight: its rows of the transposed parent
    const int64_t K = d.rows, N = d.cols;
    std::vector<char> t((size_t)N * K * es);
    CUDA_TRY(cudaMemcpy2D(t.data(), (size_t)K * es, h->dptr[root] + (size_t)P.g.coff[buf] * h->ld[root] * es,
                          (size_t)h->ld[root] * es, (size_t)K * es, N, cudaMemcpyDeviceToHost));
    char *out = static_cast<char *>(host_ptr);
    for (int64_t n = 0; n < N; ++n)
      for (int64_t k = 0; k < K; ++k) memcpy(out + (k * N + n) * es, t.data() + (n * K + k) * es, es);
    return DAG_OK;
  }
  if (P.store_t[buf]) {  // back to the caller's layout on the host
    const int64_t B = P.t_batch[buf], K = P.t_K[buf], N = P.t_N[buf];
    std::vector<char> t((size_t)B * N * K * es);
    CUDA_TRY(cudaMemcpy2D(t.data(), (size_t)K * es, h->dptr[buf], (size_t)h->ld[buf] * es, (size_t)K * es, B * N,
                          cudaMemcpyDeviceToHost));
    char *out = static_cast<char *>(host_ptr);
    for (int64_t b = 0; b < B; ++b)
      for (int64_t n = 0; n < N; ++n)
        for (int64_t k = 0; k < K; ++k)
          memcpy(out + ((b * K + k) * N + n) * es, t.data() + ((b * N + n) * K + k) * es, es);
    return DAG_OK;
  }
  CUDA_TRY(cudaMemcpy2D(host_ptr, w, h->dptr[buf], (size_t)h->ld[buf] * es, w, d.rows, cudaMemcpyDeviceToHost));
  return DAG_OK;
}

extern "C" const void *dag_device_ptr(dag_handle *h, int buf, int64_t *ld_elems) {
  if (!h || !caller_buf(h->P, buf) || h->P.store_t[h->P.g.root[buf]]) return nullptr;
  if (ld_elems) *ld_elems = h->ld[buf];
  return h->dptr[buf];
}

extern "C" dag_status dag_destroy(dag_handle *h) {
  if (!h) return DAG_OK;
  if (h->in_flight && !h->poisoned) poll_event(h->reading ? h->ev_read : h->ev_done, 10ull * 1000000000ull);
  free_handle(h);
  return DAG_OK;
}

extern "C" dag_status dag_set_device(int ordinal) {
  CUDA_TRY(cudaSetDevice(ordinal));
  return DAG_OK;
}

extern "C" void *dag_host_alloc(size_t bytes) {
  void *p = nullptr;
  if (cudaHostAlloc(&p, bytes ? bytes : 1, cudaHostAllocDefault) != cudaSuccess) {
    fail(DAG_ENOMEM, "cudaHostAlloc(%zu)", bytes);
    return nullptr;
  }
  return p;
}

extern "C" void dag_host_free(void *p) {
  if (p) cudaFreeHost(p);
}

extern "C" dag_status dag_trace_get(dag_handle *h, dag_trace_record *out, int cap, int *n) {
  if (!h || !n) return fail(DAG_EINVAL, "null argument");
  if (h->in_flight) return fail(DAG_EBUSY, "call dag_wait first");
  const int nt = (int)h->P.tiles.size();
  *n = nt;
  if (!out || cap <= 0) return DAG_OK;
  if (!h->P.opt.trace) return fail(DAG_EINVAL, "tracing was not enabled in dag_options");
  std::vector<TraceRec> tr(nt);
  if (nt) CUDA_TRY(cudaMemcpy(tr.data(), h->d_trace, (size_t)nt * sizeof(TraceRec), cudaMemcpyDeviceToHost));
  const std::vector<TileDesc> &src = h->last_mode == 0 ? h->P.queue : h->P.tiles;
  for (int i = 0; i < nt && i < cap; ++i) {
    const TileDesc &t = src[i];
    out[i] = dag_trace_record{t.node, t.r0, t.r1, t.c0, t.c1, tr[i].start_ticket, tr[i].end_ticket, tr[i].smid,
                              t.split, 0, tr[i].stamp[S_CLAIM], tr[i].stamp[S_READY], tr[i].stamp[S_WORK],
                              tr[i].stamp[S_END]};
  }
  return DAG_OK;
}

extern "C" dag_status dag_trace_launch(dag_handle *h, uint64_t *enter_exit) {
  if (!h || !enter_exit) return fail(DAG_EINVAL, "null argument");
  if (h->in_flight) return fail(DAG_EBUSY, "call dag_wait first");
  if (!h->P.opt.trace) return fail(DAG_EINVAL, "tracing was not enabled in dag_options");
  if (h->last_mode != 0) return fail(DAG_EINVAL, "the last submit was not a persistent launch");
  Ctrl c;
  CUDA_TRY(cudaMemcpy(&c, h->d_ctrl, sizeof c, cudaMemcpyDeviceToHost));
  enter_exit[0] = c.t_enter;
  enter_exit[1] = c.t_exit;
  return DAG_OK;
}

extern "C" dag_status dag_trace_stamps(dag_handle *h, uint64_t *out, int cap, int *n) {
  if (!h || !n) return fail(DAG_EINVAL, "null argument");
  if (h->in_flight) return fail(DAG_EBUSY, "call dag_wait first");
  const int nt = (int)h->P.tiles.size();
  *n = nt;
  if (!out || cap <= 0) return DAG_OK;
  if (!h->P.opt.trace) return fail(DAG_EINVAL, "tracing was not enabled in dag_options");
  std::vector<TraceRec> tr(nt);
  if (nt) CUDA_TRY(cudaMemcpy(tr.data(), h->d_trace, (size_t)nt * sizeof(TraceRec), cudaMemcpyDeviceToHost));
  for (int i = 0; i < nt && i < cap; ++i) memcpy(out + (size_t)i * kNumStamps, tr[i].stamp, sizeof tr[i].stamp);
  return DAG_OK;
}

extern "C" dag_status dag_plan_get(dag_handle *h, dag_plan_info *o) {
  if (!h || !o) return fail(DAG_EINVAL, "null argument");
  o->n_tiles = (int)h->P.tiles.size();
  o->n_counters = h->P.n_counters;
  o->n_waits = (int)h->P.waits.size();
  o->grid = h->P.grid;
  o->smem_bytes = exec_smem_bytes();
  o->flops = h->P.flops;
  o->bytes = h->P.bytes;
  o->critical_path_us = h->P.cp_us;
  o->work_bound_us = h->P.work_us;
  o->tile_override = h->P.opt.tile_override;
  o->scheduler = h->P.opt.scheduler;
  o->tuned_us = h->tuned_us;
  o->buffer_bytes = (double)h->arena_bytes;
  return DAG_OK;
}

extern "C" dag_status dag_node_costs_get(dag_handle *h, float *out, int cap, int *n) {
  if (!h || !n) return fail(DAG_EINVAL, "null argument");
  const int nn = h->P.g.nn;
  *n = nn;
  for (int i = 0; out && i < nn && i < cap; ++i) out[i] = (float)h->P.node_cost[i];
  return DAG_OK;
}

extern "C" dag_status dag_tiles_get(dag_handle *h, int32_t *out6, int cap, int *n) {
  if (!h || !n) return fail(DAG_EINVAL, "null argument");
  const int nt = (int)h->P.queue.size();
  *n = nt;
  for (int i = 0; out6 && i < nt && i < cap; ++i) {
    const TileDesc &t = h->P.queue[i];
    const int32_t r[6] = {t.node, t.r0, t.r1, t.c0, t.c1, t.cfg | (t.split << 16)};
    memcpy(out6 + 6 * i, r, sizeof r);
  }
  return DAG_OK;
}

// ---------------------------------------------------------------------------
// A whole plan serialised into one caller-provided device region.  Used by
// the entry point that allocates nothing (noalloc.cu): the region is a
// file-scope device array there, the buffers belong to the caller.
// ---------------------------------------------------------------------------
extern "C" dag_status dag_fusion_get(dag_handle *h, int32_t *out, int cap, int *n) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (!n) return fail(DAG_EINVAL, "null n");
  *n = h->P.g.nn;
  for (int v = 0; out && v < h->P.g.nn && v < cap; ++v) out[v] = h->P.absorbed_by[v];
  return DAG_OK;
}

extern "C" dag_status dag_fusion_host(const dag_node_desc *nodes, int n_nodes, const dag_edge *edges, int n_edges,
                                      const dag_buffer_desc *buffers, int n_buffers, const dag_options *opts,
                                      int32_t *out) {
  if (!out && n_nodes > 0) return fail(DAG_EINVAL, "null output array");
  Plan P;
  if (opts) P.opt = *opts;
  dag_status s = build_graph(nodes, n_nodes, edges, n_edges, buffers, n_buffers, P.g);
  if (s) return s;
  choose_merges(P);
  choose_layouts(P);
  choose_configs(P);
  choose_fusion(P);
  for (int v = 0; v < P.g.nn; ++v) out[v] = P.absorbed_by[v];
  return DAG_OK;
}

static void merge_out(const Plan &P, int32_t *leader, int32_t *col_offset, int cap) {
  for (int v = 0; v < P.g.nn && v < cap; ++v) {
    const bool m = !P.merged_into.empty() && P.merged_into[v] >= 0;
    if (leader) leader[v] = m ? P.merged_into[v] : -1;
    if (col_offset) col_offset[v] = m ? P.merge_coff[v] : 0;
  }
}

extern "C" dag_status dag_merge_get(dag_handle *h, int32_t *leader, int32_t *col_offset, int cap, int *n) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (!n) return fail(DAG_EINVAL, "null n");
  *n = h->P.g.nn;
  merge_out(h->P, leader, col_offset, cap);
  return DAG_OK;
}

extern "C" dag_status dag_merge_host(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers,
                                     int n_buffers, const dag_options *opts, int32_t *leader, int32_t *col_offset) {
  if ((!leader || !col_offset) && n_nodes > 0) return fail(DAG_EINVAL, "null output array");
  Plan P;
  if (opts) P.opt = *opts;
  dag_status s = build_graph(nodes, n_nodes, nullptr, 0, buffers, n_buffers, P.g);
  if (s) return s;
  choose_merges(P);
  merge_out(P, leader, col_offset, n_nodes);
  return DAG_OK;
}

dag_status dagx::report_error(dag_status s, const char *msg) { return fail(s, "%s", msg); }

dag_status dagx::plan_into_region(const dag_node_desc *nodes, int n_nodes, const dag_buffer_desc *buffers,
                                  int n_buffers, void *const *ptrs, const int64_t *lds, const dag_options *opts,
                                  char *region, size_t capacity, std::vector<char> &blob, ExecParams &xp,
                                  int &grid) {
  dag_status s = init_driver();
  if (s) return s;
  if (n_buffers > 0 && (!ptrs || !lds)) return fail(DAG_EINVAL, "null buffer pointer or pitch array");
  Plan P;
  if (opts) P.opt = *opts;
  if (!P.opt.timeout_ns) P.opt.timeout_ns = 2000000000ull;
  P.opt.trace = 0;
  P.opt.debug_never_ready = 0;
  P.allow_split = false;  // split K needs scratch memory
  P.allow_layout = false; // caller-owned buffers keep the caller's layout
  // every input is already in the caller's device memory: no upload flags
  std::vector<dag_buffer_desc> bufs(buffers, buffers + std::max(0, n_buffers));
  for (auto &b : bufs)
    if (b.flags & DAG_BUF_INPUT) b.flags |= DAG_BUF_RESIDENT;
  if ((s = build_graph(nodes, n_nodes, nullptr, 0, bufs.data(), n_buffers, P.g))) return s;
  Graph &g = P.g;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(DAG_EDEVICE, "no CUDA device");
  cudaDeviceGetAttribute(&P.n_sm, cudaDevAttrMultiProcessorCount, dev);
  P.grid = P.n_sm * std::max(1, max_coresident_ctas_per_sm());
  if (P.opt.max_ctas > 0) P.grid = std::min(P.grid, P.opt.max_ctas);
  plan_tiles(P);
  grid = P.grid;

  // caller buffers: root pointer and pitch; views offset into their parent
  std::vector<char *> dptr(g.nb, nullptr);
  std::vector<int64_t> ld(g.nb, 0);
  for (int b = 0; b < g.nb; ++b) {
    const int r = g.root[b];
    if (!ptrs[r]) return fail(DAG_EINVAL, "buffer %d: null device pointer", r);
    if (lds[r] < g.bufs[r].cols || (lds[r] * esize(g.bufs[r].dtype)) % 16)
      return fail(DAG_EUNSUPPORTED, "buffer %d: row pitch %lld must be >= cols and a multiple of 16 bytes", r,
                  (long long)lds[r]);
    if ((uintptr_t)ptrs[r] % 16) return fail(DAG_EUNSUPPORTED, "buffer %d: pointer not 16-byte aligned", r);
    ld[b] = lds[r];
    dptr[b] = (char *)ptrs[r] + (size_t)g.coff[b] * esize(g.bufs[b].dtype);
  }
  const int nn = g.nn, nt = (int)P.queue.size();
  std::vector<NodeParams> np(std::max(1, nn));
  std::vector<CUtensorMap> maps;
  for (int v = 0; v < nn; ++v)
    if ((s = fill_params(P, v, dptr.data(), ld.data(), np[v], maps))) return s;
  // layout inside the region; counters, flags and control block start at zero
  size_t o_maps = 0;
  size_t o_tiles = align_up(o_maps + maps.size() * sizeof(CUtensorMap), 256);
  size_t o_waits = align_up(o_tiles + (size_t)nt * sizeof(TileDesc), 256);
  size_t o_rels = align_up(o_waits + P.waits.size() * sizeof(Wait), 256);
  size_t o_nodes = align_up(o_rels + P.rels.size() * sizeof(uint32_t), 256);
  size_t o_cnt = align_up(o_nodes + np.size() * sizeof(NodeParams), 256);
  size_t o_flags = align_up(o_cnt + (size_t)std::max(1, P.n_counters) * 4, 256);
  size_t o_ctrl = align_up(o_flags + (size_t)std::max(1, P.n_flags) * 4, 256);
  size_t total = align_up(o_ctrl + sizeof(Ctrl), 256);
  if (total > capacity)
    return fail(DAG_ENOMEM, "this DAG's plan needs %zu bytes of scratch (%d tiles); the fixed scratch holds %zu bytes",
                total, nt, capacity);
  blob.assign(total, 0);
  auto put = [&](size_t o, const void *src, size_t n) { if (n) memcpy(blob.data() + o, src, n); };
  put(o_maps, maps.data(), maps.size() * sizeof(CUtensorMap));
  put(o_tiles, P.queue.data(), (size_t)nt * sizeof(TileDesc));
  put(o_waits, P.waits.data(), P.waits.size() * sizeof(Wait));
  put(o_rels, P.rels.data(), P.rels.size() * sizeof(uint32_t));
  put(o_nodes, np.data(), np.size() * sizeof(NodeParams));
  memset(&xp, 0, sizeof xp);
  xp.tiles = (const TileDesc *)(region + o_tiles);
  xp.n_tiles = nt;
  xp.waits = (const Wait *)(region + o_waits);
  xp.rels = (const uint32_t *)(region + o_rels);
  xp.nodes = (const NodeParams *)(region + o_nodes);
  xp.tmaps = (const CUtensorMap *)(region + o_maps);
  xp.counters = (uint32_t *)(region + o_cnt);
  xp.flags = (uint32_t *)(region + o_flags);
  xp.ctrl = (Ctrl *)(region + o_ctrl);
  xp.trace = nullptr;
  xp.trace_on = 0;
  xp.fused = std::any_of(P.post.begin(), P.post.end(), [](const std::vector<int> &c) { return !c.empty(); }) ? 1 : 0;
  xp.timeout_ns = P.opt.timeout_ns;
  return DAG_OK;
}

// ---------------------------------------------------------------------------
// dag_submit_cq: the paper's Alg. 1 (schedule / setup_cq / cb) on CUDA streams
// ---------------------------------------------------------------------------
namespace {

struct CqRun;
struct CqArg {
  CqRun *run;
  int kernel;
};

// State shared between the schedule loop and the host callbacks (cb).
struct CqRun {
  std::mutex mu;
  std::condition_variable cv;
  std::vector<int> comp;              // kernel -> component
  std::vector<int> end_left;          // component -> END kernels not yet finished
  std::vector<int> pred_left;         // component -> predecessor components not yet finished
  std::vector<std::vector<int>> csucc;
  std::vector<int> ready;             // the task queue F
  bool device_free = true;
  int n_done = 0, n_callbacks = 0;
  std::vector<CqArg> args;
};

void CUDART_CB cq_callback(void *p) {
  CqArg *a = static_cast<CqArg *>(p);
  CqRun *r = a->run;
  std::lock_guard<std::mutex> lk(r->mu);
  r->n_callbacks++;
  const int c = r->comp[a->kernel];
  if (--r->end_left[c] == 0) {  // T finished: release its successors and the device
    r->n_done++;
    for (int s : r->csucc[c])
      if (--r->pred_left[s] == 0) r->ready.push_back(s);
    r->device_free = true;
  }
  r->cv.notify_one();
}

}  // namespace

extern "C" dag_status dag_submit_cq(dag_handle *h, const dag_cq_options *o, dag_cq_result *res) {
  dag_status s = check_handle(h);
  if (s) return s;
  if (!o) return fail(DAG_EINVAL, "null options");
  if (h->in_flight) return fail(DAG_EBUSY, "a submit is in flight");
  if (o->n_queues < 1 || o->n_queues > 32) return fail(DAG_EINVAL, "n_queues %d not in 1..32", o->n_queues);
  if (o->components < DAG_TC_GIVEN || o->components > DAG_TC_PER_KERNEL)
    return fail(DAG_EINVAL, "bad components mode %d", o->components);
  Plan &P = h->P;
  Graph &g = P.g;
  const int n = g.nn;

  // ---- the task component partition and its graph ----
  CqRun *run = new (std::nothrow) CqRun();
  if (!run) return fail(DAG_ENOMEM, "host allocation");
  std::vector<int> raw(n);
  for (int v = 0; v < n; ++v)
    raw[v] = o->components == DAG_TC_GIVEN ? g.nodes[v].component : o->components == DAG_TC_WHOLE ? 0 : v;
  std::vector<int> ids(raw);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  const int nc = (int)ids.size();
  run->comp.resize(n);
  for (int v = 0; v < n; ++v) run->comp[v] = (int)(std::lower_bound(ids.begin(), ids.end(), raw[v]) - ids.begin());
  const std::vector<int> &comp = run->comp;
  std::vector<char> front(n, 1), end(n, 1);
  run->csucc.assign(nc, {});
  run->pred_left.assign(nc, 0);
  run->end_left.assign(nc, 0);
  for (int u = 0; u < n; ++u)
    for (int v : g.succ[u]) {
      if (comp[u] == comp[v]) { end[u] = 0; front[v] = 0; continue; }
      std::vector<int> &cs = run->csucc[comp[u]];
      if (std::find(cs.begin(), cs.end(), comp[v]) == cs.end()) { cs.push_back(comp[v]); run->pred_left[comp[v]]++; }
    }
  for (int v = 0; v < n; ++v) run->end_left[comp[v]] += end[v];
  {  // the component graph must be acyclic (a convex partition), or the schedule cannot finish
    std::vector<int> indeg(run->pred_left), stack;
    for (int c = 0; c < nc; ++c)
      if (!indeg[c]) stack.push_back(c);
    int seen = 0;
    while (!stack.empty()) {
      const int c = stack.back();
      stack.pop_back();
      ++seen;
      for (int d : run->csucc[c])
        if (--indeg[d] == 0) stack.push_back(d);
    }
    if (seen != nc) { delete run; return fail(DAG_ECYCLE, "the task components form a cycle"); }
  }
  // priority of a component: the largest bottom-level rank among its FRONT kernels
  std::vector<double> crank(nc, -1.0);
  for (int v = 0; v < n; ++v)
    if (front[v]) crank[comp[v]] = std::max(crank[comp[v]], P.rank.empty() ? 0.0 : P.rank[v]);
  std::vector<std::vector<int>> members(nc);
  for (int v : g.topo) members[comp[v]].push_back(v);

  // ---- streams and events (created once per handle) ----
  auto fail_cuda = [&](cudaError_t e) { delete run; return fail(DAG_EDEVICE, "CUDA: %s", cudaGetErrorString(e)); };
  cudaError_t ce;
  while ((int)h->cq_q.size() < o->n_queues) {
    cudaStream_t q;
    if ((ce = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking))) return fail_cuda(ce);
    h->cq_q.push_back(q);
  }
  if (!h->cq_t0) {  // the handle keeps them only once all exist (free_handle destroys the rest)
    h->cq_beg.assign(n, nullptr);
    h->cq_end.assign(n, nullptr);
    h->cq_buf.assign(g.nb, nullptr);
    for (int v = 0; v < n; ++v)
      if ((ce = cudaEventCreate(&h->cq_beg[v])) || (ce = cudaEventCreate(&h->cq_end[v]))) return fail_cuda(ce);
    for (int b = 0; b < g.nb; ++b)
      if ((ce = cudaEventCreateWithFlags(&h->cq_buf[b], cudaEventDisableTiming))) return fail_cuda(ce);
    if ((ce = cudaEventCreate(&h->cq_t0))) return fail_cuda(ce);
  }
  std::vector<char> need_up(g.nb, 0), uploaded(g.nb, 0);
  std::vector<int> up_queue(g.nb, -1);
  for (int b = 0; b < g.nb; ++b)
    need_up[b] = h->resident_dirty[b] || (P.flag_of_root[b] >= 0 && h->host_in[b]);
  ExecParams x = h->xp;
  x.tiles = h->d_coarse;
  run->args.resize(n);
  for (int v = 0; v < n; ++v) run->args[v] = CqArg{run, v};

  // ---- setup_cq + dispatch of one component ----
  std::vector<std::vector<int>> writers(g.nb);
  for (int v = 0; v < n; ++v) writers[g.root[g.nodes[v].out]].push_back(v);
  std::vector<int> writers_left(g.nb, 0);
  for (int b = 0; b < g.nb; ++b) writers_left[b] = (int)writers[b].size();
  std::vector<int> qof(n, -1), order;  // order: components in dispatch order
  std::vector<char> processed(n, 0);
  auto setup_cq = [&](int c) -> cudaError_t {
    int rr = 0;  // init(): each component's queue structure selects from q_0 on (sel_rr)
    std::vector<int> unprocessed;
    for (int v : members[c])
      if (front[v]) unprocessed.push_back(v);
    while (!unprocessed.empty()) {
      // the unprocessed kernel with the largest bottom-level rank (ties: topological order)
      size_t pick = 0;
      for (size_t i = 1; i < unprocessed.size(); ++i) {
        const int a = unprocessed[i], b = unprocessed[pick];
        const double ra = P.rank.empty() ? 0.0 : P.rank[a], rb = P.rank.empty() ? 0.0 : P.rank[b];
        if (ra > rb || (ra == rb && g.topo_pos[a] < g.topo_pos[b])) pick = i;
      }
      const int k = unprocessed[pick];
      unprocessed.erase(unprocessed.begin() + pick);
      const int qi = rr++ % o->n_queues;
      cudaStream_t q = h->cq_q[qi];
      cudaError_t e;
      // writes: isolated inputs of k (once per run), on k's queue
      int in[3];
      const int ni = g.inputs(k, in);
      for (int i = 0; i < ni; ++i) {
        const int b = g.root[in[i]];
        if (need_up[b] && !uploaded[b]) {
          if ((e = copy_h2d(h, b, q)) || (e = cudaEventRecord(h->cq_buf[b], q))) return e;
          uploaded[b] = 1;
          up_queue[b] = qi;
        } else if (uploaded[b] && up_queue[b] != qi) {
          if ((e = cudaStreamWaitEvent(q, h->cq_buf[b], 0))) return e;
        }
      }
      // E_Q: predecessors inside T on other queues
      for (int u : g.pred[k])
        if (comp[u] == c && qof[u] != qi)
          if ((e = cudaStreamWaitEvent(q, h->cq_end[u], 0))) return e;
      // ndrange
      if ((e = cudaEventRecord(h->cq_beg[k], q))) return e;
      if (launch_in_turn(P, k) >= 0 && (e = launch_node_coarse(x, P, launch_in_turn(P, k), q))) return e;
      if ((e = cudaEventRecord(h->cq_end[k], q))) return e;
      qof[k] = qi;
      processed[k] = 1;
      // read: a registered output, once its last writer is enqueued (writers of
      // a root's column views on other queues of T are waited for; those of
      // earlier components have finished)
      const int ob = g.root[g.nodes[k].out];
      if (h->host_out[ob] && --writers_left[ob] == 0) {
        for (int u : writers[ob])
          if (u != k && comp[u] == c && qof[u] != qi)
            if ((e = cudaStreamWaitEvent(q, h->cq_end[u], 0))) return e;
        const dag_buffer_desc &d = g.bufs[ob];
        const size_t w = (size_t)d.cols * esize(d.dtype);
        if ((e = cudaMemcpy2DAsync(h->host_out[ob], w, h->dptr[ob], (size_t)h->ld[ob] * esize(d.dtype), w, d.rows,
                                   cudaMemcpyDeviceToHost, q)))
          return e;
      }
      if (end[k] && (e = cudaLaunchHostFunc(q, cq_callback, &run->args[k]))) return e;
      // successors in T whose predecessors in T are all processed
      for (int w : g.succ[k]) {
        if (comp[w] != c || processed[w] ||
            std::find(unprocessed.begin(), unprocessed.end(), w) != unprocessed.end())
          continue;
        bool ok = true;
        for (int u : g.pred[w]) ok &= comp[u] != c || processed[u];
        if (ok) unprocessed.push_back(w);
      }
    }
    return cudaSuccess;
  };

  // ---- schedule ----
  if ((ce = cudaEventRecord(h->cq_t0, h->cq_q[0]))) return fail_cuda(ce);
  for (int i = 1; i < o->n_queues; ++i)
    if ((ce = cudaStreamWaitEvent(h->cq_q[i], h->cq_t0, 0))) return fail_cuda(ce);
  const auto t_host0 = std::chrono::steady_clock::now();
  const uint64_t limit = o->timeout_ns ? o->timeout_ns : 10000000000ull;
  {
    std::unique_lock<std::mutex> lk(run->mu);
    for (int c = 0; c < nc; ++c)
      if (!run->pred_left[c]) run->ready.push_back(c);
    while (run->n_done < nc) {
      while (run->device_free && !run->ready.empty()) {
        size_t pick = 0;
        for (size_t i = 1; i < run->ready.size(); ++i) {
          const int a = run->ready[i], b = run->ready[pick];
          if (o->fifo ? a < b : (crank[a] > crank[b] || (crank[a] == crank[b] && a < b))) pick = i;
        }
        const int c = run->ready[pick];
        run->ready.erase(run->ready.begin() + pick);
        run->device_free = false;
        order.push_back(c);
        lk.unlock();
        const cudaError_t e = setup_cq(c);
        lk.lock();
        if (e) {
          lk.unlock();
          for (cudaStream_t q : h->cq_q) cudaStreamSynchronize(q);  // callbacks already enqueued finish
          h->poisoned = DAG_EDEVICE;
          return fail(DAG_EDEVICE, "setup_cq: %s", cudaGetErrorString(e));  // run leaked: callbacks may hold it
        }
      }
      if (run->n_done == nc) break;
      if (!run->cv.wait_for(lk, std::chrono::nanoseconds(limit),
                            [&] { return run->n_done == nc || (run->device_free && !run->ready.empty()); })) {
        h->poisoned = DAG_ETIMEOUT;
        return fail(DAG_ETIMEOUT, "no callback within the limit");  // run leaked: callbacks may still come
      }
    }
  }
  const double host_us =
      std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t_host0).count();
  for (cudaStream_t q : h->cq_q)
    if ((ce = cudaStreamSynchronize(q))) {
      h->poisoned = DAG_EDEVICE;
      delete run;
      return fail(DAG_EDEVICE, "device error: %s", cudaGetErrorString(ce));
    }
  for (int b = 0; b < g.nb; ++b)
    if (uploaded[b] && (g.bufs[b].flags & DAG_BUF_RESIDENT)) h->resident_dirty[b] = 0;

  // ---- timings ----
  std::vector<float> t_beg(n, 0.f), t_end(n, 0.f);
  double dev = 0.0;
  for (int v = 0; v < n; ++v) {
    cudaEventElapsedTime(&t_beg[v], h->cq_t0, h->cq_beg[v]);
    cudaEventElapsedTime(&t_end[v], h->cq_t0, h->cq_end[v]);
    t_beg[v] *= 1000.f;
    t_end[v] *= 1000.f;
    dev = std::max(dev, (double)t_end[v]);
    if (o->node_start_us) o->node_start_us[v] = t_beg[v];
    if (o->node_end_us) o->node_end_us[v] = t_end[v];
    if (o->node_queue) o->node_queue[v] = qof[v];
  }
  double gap = 0.0;
  for (size_t i = 1; i < order.size(); ++i) {
    double last_end = 0.0, first_beg = 1e30;
    for (int v : members[order[i - 1]]) last_end = std::max(last_end, (double)t_end[v]);
    for (int v : members[order[i]]) first_beg = std::min(first_beg, (double)t_beg[v]);
    gap += std::max(0.0, first_beg - last_end);
  }
  if (res) {
    res->device_us = dev;
    res->host_us = host_us;
    res->gap_us = gap;
    res->n_components = nc;
    res->n_callbacks = run->n_callbacks;
  }
  delete run;
  return DAG_OK;
}
