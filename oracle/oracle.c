/*
 * oracle.c -- plain, slow, FP64 CPU executor for application DAGs.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call, link or
 * execute this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * What it computes (the paper's problem statement, §3 "Problem Formulation"):
 * an application DAG G = <(K,B),(E_I,E_O,E)> of data-parallel kernels K over
 * buffers B, executed in a topologically sorted order (Def. 5, valid
 * schedule).  Each kernel reads input buffers and writes one output buffer
 * (§1, fork-join example; §2 vadd example).  Kernel semantics:
 *
 *   GEMM     C = act(scale * A.B + bias)      A is MxK, B is KxN, row-major,
 *            as in the matmul kernel of §4.A (globalWorkSize = [M,N,1]);
 *            trans_b: B stored NxK; batch: row-stacked independent problems
 *            (the per-sequence QK^T and PV products of the §5 head DAG).
 *   ADD      C = act(A + B)                   (vadd, §2; join K3 of §1)
 *   SOFTMAX  y_ij = exp(s x_ij - m_i) / sum_j exp(s x_ij - m_i),
 *            m_i = max_j s x_ij               (B = Softmax(A), §5)
 *   UNARY    C = act(A)
 *   act: none | relu max(0,x) | gelu 0.5 x (1 + erf(x / sqrt 2))
 *
 * All arithmetic is double; sums over k run in increasing k.  Inputs are read
 * as stored (f32 or bf16 bits) and results are rounded once to the output
 * buffer's dtype, round-to-nearest-even (f64->f32 by the C cast, f64->bf16 by
 * the exact power-of-two scaling in or_f64_to_bf16 below).
 *
 * Also here: a tiled simulator (same per-element arithmetic, a region at a
 * time, in any caller-given tile order) and a trace checker that decides, from
 * each tile's read and write regions alone, whether an observed execution was
 * dependency-legal (Def. 5 lifted from kernels to tiles).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_F32 = 0, OR_BF16 = 1 };
enum { OR_GEMM = 0, OR_ADD = 1, OR_SOFTMAX = 2, OR_UNARY = 3 };
enum { OR_ACT_NONE = 0, OR_ACT_RELU = 1, OR_ACT_GELU = 2 };
enum {
  OR_OK = 0, OR_EINVAL = 1, OR_ECYCLE = 2, OR_ESHAPE = 3, OR_EDTYPE = 4,
  OR_EMULTIWRITER = 5, OR_ENOMEM = 6
};

typedef struct { int32_t rows, cols, dtype, view_of, col_offset; } or_buffer;
typedef struct { int32_t op, a, b, bias, out, trans_b, act, batch; double scale; } or_node;
/* a tile: rows [r0,r1) x cols [c0,c1) of its node's output buffer (view coordinates) */
typedef struct { int32_t node, r0, r1, c0, c1; } or_tile;
/* a region of a physical (root) buffer */
typedef struct { int32_t root, r0, r1, c0, c1; } or_region;

/* ------------------------------------------------------------------ */
/* storage                                                              */
/* ------------------------------------------------------------------ */
static double load_bf16(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

/* f64 -> bf16, round to nearest even.  bf16 keeps 8 significant bits and the
 * f32 exponent range: the representable neighbours of |x| in binade 2^E are the
 * multiples of 2^(E-7) (2^-133 below the normal range), so scale by that power
 * of two (exact), round to an integer with ties to even (rint under the
 * default rounding mode), and scale back. */
uint16_t or_f64_to_bf16(double x) {
  if (isnan(x)) return 0x7FC0;
  int neg = signbit(x) ? 1 : 0;
  double a = fabs(x);
  double v;
  if (a == 0.0) {
    v = 0.0;
  } else if (isinf(a)) {
    v = INFINITY;
  } else {
    int e;
    frexp(a, &e);             /* a = f * 2^e, f in [0.5,1): binade exponent E = e-1 */
    int E = e - 1;
    if (E < -126) E = -126;   /* subnormal spacing 2^-133 */
    double q = ldexp(a, 7 - E);
    q = rint(q);
    v = ldexp(q, E - 7);
    if (v >= ldexp(1.0, 128)) v = INFINITY;
  }
  float f = (float)v;         /* exact: v is a bf16 value */
  uint32_t u;
  memcpy(&u, &f, 4);
  uint16_t h = (uint16_t)(u >> 16);
  if (neg) h |= 0x8000;
  return h;
}

typedef struct {
  char *base;      /* root storage */
  int64_t ld;      /* elements per row of the root */
  int64_t coff;    /* column offset of this view in the root */
  int dtype;
} acc_t;

static acc_t accessor(const or_buffer *B, void *const *data, int id) {
  acc_t a;
  int root = id;
  int64_t coff = 0;
  while (B[root].view_of >= 0) { coff += B[root].col_offset; root = B[root].view_of; }
  a.base = (char *)data[root];
  a.ld = B[root].cols;
  a.coff = coff;
  a.dtype = B[root].dtype;
  return a;
}

static inline double get(const acc_t *a, int64_t r, int64_t c) {
  int64_t i = r * a->ld + a->coff + c;
  if (a->dtype == OR_F32) return (double)((const float *)a->base)[i];
  return load_bf16(((const uint16_t *)a->base)[i]);
}

static inline void put(const acc_t *a, int64_t r, int64_t c, double v) {
  int64_t i = r * a->ld + a->coff + c;
  if (a->dtype == OR_F32) ((float *)a->base)[i] = (float)v;
  else ((uint16_t *)a->base)[i] = or_f64_to_bf16(v);
}

/* ------------------------------------------------------------------ */
/* kernel semantics                                                     */
/* ------------------------------------------------------------------ */
static double activate(int act, double x) {
  switch (act) {
    case OR_ACT_RELU: return x < 0.0 ? 0.0 : x;   /* NaN passes through */
    case OR_ACT_GELU: return 0.5 * x * (1.0 + erf(x / sqrt(2.0)));
    default: return x;
  }
}

/* per-batch GEMM dimensions from the operand shapes */
static void gemm_dims(const or_buffer *B, const or_node *n, int64_t *M, int64_t *N, int64_t *K) {
  *M = B[n->a].rows / n->batch;
  *K = B[n->a].cols;
  *N = n->trans_b ? B[n->b].rows / n->batch : B[n->b].cols;
}

/* write rows [r0,r1) x cols [c0,c1) of node n's output */
static int run_region(const or_buffer *Bf, void *const *data, const or_node *n,
                       int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  acc_t O = accessor(Bf, data, n->out);
  acc_t A = accessor(Bf, data, n->a);
  if (n->op == OR_GEMM) {
    /* C[r][j] = act(scale * sum_{k=0}^{K-1} A[r][k] * B(k,j) + bias[j]), the sum
     * accumulated in increasing k for every element.  The B operand of the
     * current batch is widened to double once (bp[k][j]); the k loop sits
     * outside the j loop, which changes no element's sequence of operations. */
    acc_t Bm = accessor(Bf, data, n->b);
    acc_t bias;
    if (n->bias >= 0) bias = accessor(Bf, data, n->bias);
    int64_t M, N, K;
    gemm_dims(Bf, n, &M, &N, &K);
    int64_t w = c1 - c0;
    double *bp = malloc(sizeof(double) * (size_t)(K * w + 1));
    double *acc = malloc(sizeof(double) * (size_t)(w + 1));
    if (!bp || !acc) { free(bp); free(acc); return OR_ENOMEM; }
    int64_t cur = -1;
    for (int64_t r = r0; r < r1; ++r) {
      int64_t bt = r / M;
      if (bt != cur) {
        for (int64_t k = 0; k < K; ++k)
          for (int64_t j = 0; j < w; ++j)
            bp[k * w + j] = n->trans_b ? get(&Bm, bt * N + c0 + j, k) : get(&Bm, bt * K + k, c0 + j);
        cur = bt;
      }
      for (int64_t j = 0; j < w; ++j) acc[j] = 0.0;
      for (int64_t k = 0; k < K; ++k) {
        double a = get(&A, r, k);
        const double *row = bp + k * w;
        for (int64_t j = 0; j < w; ++j) acc[j] += a * row[j];
      }
      for (int64_t j = 0; j < w; ++j) {
        double v = n->scale * acc[j];
        if (n->bias >= 0) v += get(&bias, 0, c0 + j);
        put(&O, r, c0 + j, activate(n->act, v));
      }
    }
    free(bp);
    free(acc);
  } else if (n->op == OR_ADD) {
    acc_t Bm = accessor(Bf, data, n->b);
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t j = c0; j < c1; ++j)
        put(&O, r, j, activate(n->act, get(&A, r, j) + get(&Bm, r, j)));
  } else if (n->op == OR_UNARY) {
    for (int64_t r = r0; r < r1; ++r)
      for (int64_t j = c0; j < c1; ++j) put(&O, r, j, activate(n->act, get(&A, r, j)));
  } else { /* SOFTMAX: statistics over the whole row, then the requested columns */
    int64_t N = Bf[n->a].cols;
    for (int64_t r = r0; r < r1; ++r) {
      double m = -INFINITY;
      int nan = 0;
      for (int64_t j = 0; j < N; ++j) {
        double x = n->scale * get(&A, r, j);
        if (isnan(x)) nan = 1;
        if (x > m) m = x;
      }
      double s = 0.0;
      for (int64_t j = 0; j < N; ++j) s += exp(n->scale * get(&A, r, j) - m);
      for (int64_t j = c0; j < c1; ++j) {
        double y = exp(n->scale * get(&A, r, j) - m) / s;
        put(&O, r, j, nan ? NAN : y);
      }
    }
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* regions and dependencies                                             */
/* ------------------------------------------------------------------ */
static or_region phys(const or_buffer *B, int id, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
  int root = id;
  int64_t off = 0;
  while (B[root].view_of >= 0) { off += B[root].col_offset; root = B[root].view_of; }
  or_region g = {root, (int32_t)r0, (int32_t)r1, (int32_t)(c0 + off), (int32_t)(c1 + off)};
  return g;
}

static int overlap(const or_region *x, const or_region *y) {
  return x->root == y->root && x->r0 < y->r1 && y->r0 < x->r1 && x->c0 < y->c1 && y->c0 < x->c1;
}

/* the physical regions a tile reads (returns count, at most 3) */
int or_tile_reads(const or_buffer *B, const or_node *nodes, const or_tile *t, or_region *out) {
  const or_node *n = &nodes[t->node];
  int k = 0;
  if (n->op == OR_GEMM) {
    int64_t M, N, K;
    gemm_dims(B, n, &M, &N, &K);
    int64_t bt = t->r0 / M;
    out[k++] = phys(B, n->a, t->r0, t->r1, 0, K);
    if (n->trans_b) out[k++] = phys(B, n->b, bt * N + t->c0, bt * N + t->c1, 0, K);
    else out[k++] = phys(B, n->b, bt * K, bt * K + K, t->c0, t->c1);
    if (n->bias >= 0) out[k++] = phys(B, n->bias, 0, 1, t->c0, t->c1);
  } else if (n->op == OR_SOFTMAX) {
    out[k++] = phys(B, n->a, t->r0, t->r1, 0, B[n->a].cols);
  } else {
    out[k++] = phys(B, n->a, t->r0, t->r1, t->c0, t->c1);
    if (n->op == OR_ADD) out[k++] = phys(B, n->b, t->r0, t->r1, t->c0, t->c1);
  }
  return k;
}

or_region or_tile_write(const or_buffer *B, const or_node *nodes, const or_tile *t) {
  return phys(B, nodes[t->node].out, t->r0, t->r1, t->c0, t->c1);
}

/* ------------------------------------------------------------------ */
/* validation and topological order                                     */
/* ------------------------------------------------------------------ */
static int valid_id(int id, int nb) { return id >= 0 && id < nb; }

int or_validate(const or_buffer *B, int nb, const or_node *nodes, int nn) {
  for (int i = 0; i < nb; ++i) {
    if (B[i].rows <= 0 || B[i].cols <= 0) return OR_ESHAPE;
    if (B[i].dtype != OR_F32 && B[i].dtype != OR_BF16) return OR_EDTYPE;
    if (B[i].view_of >= 0) {
      const or_buffer *p;
      if (!valid_id(B[i].view_of, nb) || B[i].view_of == i) return OR_EINVAL;
      p = &B[B[i].view_of];
      if (p->view_of >= 0) return OR_EINVAL;                 /* one level of views */
      if (p->rows != B[i].rows || B[i].col_offset < 0 || B[i].col_offset + B[i].cols > p->cols)
        return OR_ESHAPE;
      if (p->dtype != B[i].dtype) return OR_EDTYPE;
    }
  }
  for (int v = 0; v < nn; ++v) {
    const or_node *n = &nodes[v];
    if (!valid_id(n->a, nb) || !valid_id(n->out, nb)) return OR_EINVAL;
    if (n->act < OR_ACT_NONE || n->act > OR_ACT_GELU) return OR_EINVAL;
    const or_buffer *A = &B[n->a], *O = &B[n->out];
    if (n->op == OR_GEMM) {
      if (!valid_id(n->b, nb) || n->batch < 1) return OR_EINVAL;
      const or_buffer *Bm = &B[n->b];
      if (A->rows % n->batch || Bm->rows % n->batch) return OR_ESHAPE;
      int64_t M, N, K;
      gemm_dims(B, n, &M, &N, &K);
      int64_t Kb = n->trans_b ? Bm->cols : Bm->rows / n->batch;
      if (Kb != K || O->rows != A->rows || O->cols != N) return OR_ESHAPE;
      if (n->bias >= 0) {
        if (!valid_id(n->bias, nb)) return OR_EINVAL;
        if (B[n->bias].rows != 1 || B[n->bias].cols != N) return OR_ESHAPE;
      }
    } else if (n->op == OR_ADD) {
      if (!valid_id(n->b, nb)) return OR_EINVAL;
      if (B[n->b].rows != O->rows || B[n->b].cols != O->cols || A->rows != O->rows || A->cols != O->cols)
        return OR_ESHAPE;
    } else if (n->op == OR_SOFTMAX || n->op == OR_UNARY) {
      if (A->rows != O->rows || A->cols != O->cols) return OR_ESHAPE;
    } else {
      return OR_EINVAL;
    }
  }
  /* single writer per physical element; no kernel reads what it writes */
  for (int u = 0; u < nn; ++u) {
    or_region wu = phys(B, nodes[u].out, 0, B[nodes[u].out].rows, 0, B[nodes[u].out].cols);
    for (int v = 0; v < nn; ++v) {
      if (v != u) {
        or_region wv = phys(B, nodes[v].out, 0, B[nodes[v].out].rows, 0, B[nodes[v].out].cols);
        if (overlap(&wu, &wv)) return OR_EMULTIWRITER;
      }
      const or_node *n = &nodes[v];
      int ins[3] = {n->a, n->b, n->bias};
      for (int q = 0; q < 3; ++q) {
        if (ins[q] < 0) continue;
        or_region r = phys(B, ins[q], 0, B[ins[q]].rows, 0, B[ins[q]].cols);
        if (v == u && overlap(&wu, &r)) return OR_EMULTIWRITER;  /* in-place */
      }
    }
  }
  return OR_OK;
}

/* node u precedes node v when v reads a region u writes (E_O then E then E_I) */
static int node_edge(const or_buffer *B, const or_node *nodes, int u, int v) {
  if (u == v) return 0;
  or_region w = phys(B, nodes[u].out, 0, B[nodes[u].out].rows, 0, B[nodes[u].out].cols);
  const or_node *n = &nodes[v];
  int ins[3] = {n->a, n->b, n->bias};
  for (int q = 0; q < 3; ++q) {
    if (ins[q] < 0) continue;
    or_region r = phys(B, ins[q], 0, B[ins[q]].rows, 0, B[ins[q]].cols);
    if (overlap(&w, &r)) return 1;
  }
  return 0;
}

/* Kahn's algorithm, ties broken by the smallest kernel id */
int or_topo_order(const or_buffer *B, int nb, const or_node *nodes, int nn, int32_t *order) {
  (void)nb;
  int *indeg = calloc((size_t)nn + 1, sizeof(int));
  char *done = calloc((size_t)nn + 1, 1);
  if (!indeg || !done) { free(indeg); free(done); return OR_ENOMEM; }
  for (int u = 0; u < nn; ++u)
    for (int v = 0; v < nn; ++v) indeg[v] += node_edge(B, nodes, u, v);
  int rc = OR_OK;
  for (int pos = 0; pos < nn; ++pos) {
    int pick = -1;
    for (int v = 0; v < nn; ++v)
      if (!done[v] && indeg[v] == 0) { pick = v; break; }
    if (pick < 0) { rc = OR_ECYCLE; break; }
    done[pick] = 1;
    order[pos] = pick;
    for (int v = 0; v < nn; ++v) indeg[v] -= node_edge(B, nodes, pick, v);
  }
  free(indeg);
  free(done);
  return rc;
}

/* is `order` a topological order of the kernel DAG? */
int or_is_topological(const or_buffer *B, const or_node *nodes, int nn, const int32_t *order) {
  int *pos = malloc(sizeof(int) * ((size_t)nn + 1));
  if (!pos) return 0;
  for (int i = 0; i < nn; ++i) pos[i] = -1;
  for (int i = 0; i < nn; ++i) {
    if (order[i] < 0 || order[i] >= nn || pos[order[i]] >= 0) { free(pos); return 0; }
    pos[order[i]] = i;
  }
  int ok = 1;
  for (int u = 0; u < nn && ok; ++u)
    for (int v = 0; v < nn && ok; ++v)
      if (node_edge(B, nodes, u, v) && pos[u] > pos[v]) ok = 0;
  free(pos);
  return ok;
}

/* ------------------------------------------------------------------ */
/* executors                                                            */
/* ------------------------------------------------------------------ */
/* Run every kernel in `order` (NULL: Kahn order).  data[i] holds root buffer i
 * densely (ld = cols); inputs are read from it and outputs written into it. */
int or_run(const or_buffer *B, int nb, const or_node *nodes, int nn, void *const *data,
           const int32_t *order) {
  int rc = or_validate(B, nb, nodes, nn);
  if (rc) return rc;
  int32_t *ord = malloc(sizeof(int32_t) * ((size_t)nn + 1));
  if (!ord) return OR_ENOMEM;
  if (order) {
    if (!or_is_topological(B, nodes, nn, order)) { free(ord); return OR_EINVAL; }
    memcpy(ord, order, sizeof(int32_t) * (size_t)nn);
  } else if ((rc = or_topo_order(B, nb, nodes, nn, ord)) != OR_OK) {
    free(ord);
    return rc;
  }
  for (int i = 0; i < nn; ++i) {
    const or_node *n = &nodes[ord[i]];
    if ((rc = run_region(B, data, n, 0, B[n->out].rows, 0, B[n->out].cols)) != OR_OK) break;
  }
  free(ord);
  return rc;
}

/* Run one kernel only (used to time a bounded sample). */
int or_run_node(const or_buffer *B, int nb, const or_node *nodes, int nn, void *const *data, int k,
                int64_t r0, int64_t r1) {
  if (k < 0 || k >= nn) return OR_EINVAL;
  (void)nb;
  const or_node *n = &nodes[k];
  if (r1 > B[n->out].rows) r1 = B[n->out].rows;
  return run_region(B, data, n, r0, r1, 0, B[n->out].cols);
}

/* Tiled simulator: run tiles[order[i]] in sequence, each writing its region
 * only.  No dependency is checked here; reading a region nobody has written
 * yet reads whatever the caller left there (tests poison it with NaN). */
int or_run_tiles(const or_buffer *B, int nb, const or_node *nodes, int nn, void *const *data,
                 const or_tile *tiles, int nt, const int32_t *order) {
  (void)nb;
  for (int i = 0; i < nt; ++i) {
    const or_tile *t = &tiles[order ? order[i] : i];
    if (t->node < 0 || t->node >= nn) return OR_EINVAL;
    int rc = run_region(B, data, &nodes[t->node], t->r0, t->r1, t->c0, t->c1);
    if (rc) return rc;
  }
  return OR_OK;
}

/* A plain tiling of every kernel: GEMM tiles bm x bn within one batch; softmax
 * tiles of bm full rows; add/unary tiles bm x bn.  Returns the tile count, or
 * -1 when cap is too small. */
int or_make_tiles(const or_buffer *B, const or_node *nodes, int nn, int bm, int bn, or_tile *out, int cap) {
  int k = 0;
  for (int v = 0; v < nn; ++v) {
    const or_node *n = &nodes[v];
    int64_t R = B[n->out].rows, C = B[n->out].cols;
    int64_t M = R, step_c = bn;
    if (n->op == OR_GEMM) M = R / n->batch;
    if (n->op == OR_SOFTMAX) step_c = C;
    for (int64_t base = 0; base < R; base += M)
      for (int64_t r = base; r < base + M; r += bm)
        for (int64_t c = 0; c < C; c += step_c) {
          if (k >= cap) return -1;
          or_tile t = {v, (int32_t)r, (int32_t)(r + bm < base + M ? r + bm : base + M), (int32_t)c,
                       (int32_t)(c + step_c < C ? c + step_c : C)};
          out[k++] = t;
        }
  }
  return k;
}

/* tile edges u -> v (v reads what u writes); returns count, or -1 past cap */
int or_tile_deps(const or_buffer *B, const or_node *nodes, const or_tile *tiles, int nt, int32_t *edges,
                 int cap) {
  int k = 0;
  for (int u = 0; u < nt; ++u) {
    or_region w = or_tile_write(B, nodes, &tiles[u]);
    for (int v = 0; v < nt; ++v) {
      if (u == v) continue;
      or_region rd[3];
      int nr = or_tile_reads(B, nodes, &tiles[v], rd);
      for (int q = 0; q < nr; ++q)
        if (overlap(&w, &rd[q])) {
          if (k >= cap) return -1;
          edges[2 * k] = u;
          edges[2 * k + 1] = v;
          ++k;
          break;
        }
    }
  }
  return k;
}

/* ------------------------------------------------------------------ */
/* trace checker                                                        */
/* ------------------------------------------------------------------ */
/* Decide whether an observed execution was legal.  Each tile carries the
 * ticket it drew after acquiring its inputs (start) and the ticket it drew
 * after writing its output and before releasing it (end), both from one
 * global counter.  Legal iff
 *   (1) every kernel's output is covered by its tiles exactly once,
 *   (2) start < end for every tile, and
 *   (3) end(u) < start(v) whenever v reads a region u writes.
 * Returns 0 if legal; otherwise 1 (coverage), 2 (start >= end) or 3 (order),
 * with the offending tiles in *bad_u / *bad_v. */
int or_check_trace(const or_buffer *B, int nb, const or_node *nodes, int nn, const or_tile *tiles, int nt,
                   const uint32_t *start, const uint32_t *end, int32_t *bad_u, int32_t *bad_v) {
  *bad_u = *bad_v = -1;
  /* (1) coverage, per kernel */
  for (int v = 0; v < nn; ++v) {
    int64_t R = B[nodes[v].out].rows, C = B[nodes[v].out].cols;
    unsigned char *cnt = calloc((size_t)(R * C), 1);
    if (!cnt) return OR_ENOMEM + 100;
    int bad = 0;
    for (int t = 0; t < nt && !bad; ++t) {
      if (tiles[t].node != v) continue;
      const or_tile *x = &tiles[t];
      if (x->r0 < 0 || x->r1 > R || x->c0 < 0 || x->c1 > C || x->r0 >= x->r1 || x->c0 >= x->c1) {
        bad = 1; *bad_u = t; break;
      }
      for (int64_t r = x->r0; r < x->r1 && !bad; ++r)
        for (int64_t c = x->c0; c < x->c1; ++c)
          if (++cnt[r * C + c] > 1) { bad = 1; *bad_u = t; break; }
    }
    for (int64_t i = 0; i < R * C && !bad; ++i)
      if (cnt[i] != 1) { bad = 1; *bad_v = v; }
    free(cnt);
    if (bad) return 1;
  }
  /* (2) */
  for (int t = 0; t < nt; ++t)
    if (!(start[t] < end[t])) { *bad_u = t; return 2; }
  /* (3) writers indexed by physical buffer */
  int *head = malloc(sizeof(int) * ((size_t)nb + 1));
  int *next = malloc(sizeof(int) * ((size_t)nt + 1));
  or_region *wr = malloc(sizeof(or_region) * ((size_t)nt + 1));
  if (!head || !next || !wr) { free(head); free(next); free(wr); return OR_ENOMEM + 100; }
  for (int i = 0; i < nb; ++i) head[i] = -1;
  for (int u = 0; u < nt; ++u) {
    wr[u] = or_tile_write(B, nodes, &tiles[u]);
    next[u] = head[wr[u].root];
    head[wr[u].root] = u;
  }
  int rc = 0;
  for (int v = 0; v < nt && !rc; ++v) {
    or_region rd[3];
    int nr = or_tile_reads(B, nodes, &tiles[v], rd);
    for (int q = 0; q < nr && !rc; ++q)
      for (int u = head[rd[q].root]; u >= 0; u = next[u])
        if (u != v && overlap(&wr[u], &rd[q]) && !(end[u] < start[v])) {
          *bad_u = u; *bad_v = v; rc = 3; break;
        }
  }
  free(head);
  free(next);
  free(wr);
  return rc;
}
