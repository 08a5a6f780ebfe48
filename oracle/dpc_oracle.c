/*
 * CPU oracle for the consolidated dynamic-parallelism hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or load
 * this file; only the tests, the package's smoke check and the benchmark's CPU
 * baseline do. It shares no code, header or constant with the CUDA library.
 *
 * Plain, single-threaded, obviously-correct C. Each function states the passage
 * of Wu, Li & Becchi, "Compiler-Assisted Workload Consolidation for Efficient
 * Dynamic Parallelism on GPU" (arXiv 1606.08150) it follows:
 *
 *   oracle_sssp_dijkstra      single-source shortest paths (Sec. III.A, Fig. 1b:
 *                             the SSSP kernel; the result is the unique
 *                             shortest-path distance, computed by Dijkstra)
 *   oracle_sssp_frontier      the same distances by frontier rounds of edge
 *                             relaxation (Fig. 1b applied round after round),
 *                             with per-round frontier sizes and the number of
 *                             frontier vertices above THRESHOLD (the per-thread
 *                             child launches of basic-DP)
 *   oracle_sssp_nearfar       the frontier rounds with a near-far split of the
 *                             vertices that dropped (near: relaxed next round;
 *                             far: kept until the split distance passes them),
 *                             after Davidson et al., IPDPS 2014
 *   oracle_spmv_f64           y = A x for CSR A in double precision (Sec. V,
 *                             SpMV benchmark; irregular loop of Sec. II.B)
 *   oracle_tree_descendants   number of proper descendants of every node
 *                             (Sec. V, tree descendants; recursion of Fig. 1c)
 *   oracle_tree_height        height of every node, leaves 0 (Sec. V, tree heights)
 *   oracle_tree_levels        per-depth counts of nodes, internal nodes and
 *                             child edges (the recursion levels of Fig. 1c)
 *   oracle_pagerank           PageRank by power iteration (Sec. V, the PR
 *                             benchmark): rank pushed along out-edges, damping,
 *                             uniform teleport, dangling mass spread uniformly
 *   oracle_bfs                hop distance from a source by a FIFO queue
 *                             (Sec. V, BFS-Rec: the levels its recursion
 *                             settles on; unique, so any traversal order works)
 *   oracle_color_jp           graph colouring by round sweep (Sec. V,
 *                             the GC benchmark): in round r every uncoloured
 *                             vertex whose priority beats all its uncoloured
 *                             neighbours takes colour r
 *   oracle_consolidation_launches
 *                             child-kernel launches of one parent grid at each
 *                             consolidation granularity (Sec. IV.B): one per
 *                             buffered item (basic-DP), per warp, per block and
 *                             per grid holding at least one buffered item
 *
 * Parity pins for every function live in the CPU tests (Floyd-Warshall, dense
 * matrix-vector products, brute-force ancestor walks, hand-worked examples).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF 0xFFFFFFFFu

/* ------------------------------------------------------------------ SSSP */

typedef struct { uint64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *sz, heap_item it) {
  int64_t i = (*sz)++;
  h[i] = it;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= h[i].d) break;
    heap_item t = h[p]; h[p] = h[i]; h[i] = t;
    i = p;
  }
}

static heap_item heap_pop(heap_item *h, int64_t *sz) {
  heap_item top = h[0];
  h[0] = h[--(*sz)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < *sz && h[l].d < h[s].d) s = l;
    if (r < *sz && h[r].d < h[s].d) s = r;
    if (s == i) break;
    heap_item t = h[s]; h[s] = h[i]; h[i] = t;
    i = s;
  }
  return top;
}

/*
 * Dijkstra with a binary heap and lazy deletion. Distances are accumulated in
 * 64 bits; unreachable vertices get 0xFFFFFFFF. Self-loops never shorten a
 * path and duplicate edges simply compete. Returns 0, 1 if some finite
 * distance does not fit below 0xFFFFFFFF, -1 on bad arguments.
 */
int oracle_sssp_dijkstra(int32_t n, const int32_t *off, const int32_t *col, const uint32_t *w, int32_t source,
                         uint32_t *dist_out) {
  if (n < 1 || source < 0 || source >= n) return -1;
  uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint8_t *done = (uint8_t *)calloc((size_t)n, 1);
  int64_t m = off[n];
  heap_item *h = (heap_item *)malloc((size_t)(m + 1) * sizeof(heap_item));
  if (!d || !done || !h) { free(d); free(done); free(h); return -1; }
  for (int32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  int64_t sz = 0;
  d[source] = 0;
  heap_push(h, &sz, (heap_item){0, source});
  while (sz > 0) {
    heap_item it = heap_pop(h, &sz);
    int32_t u = it.v;
    if (done[u] || it.d != d[u]) continue;
    done[u] = 1;
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      int32_t v = col[e];
      uint64_t nd = d[u] + (uint64_t)w[e];
      if (nd < d[v]) {
        d[v] = nd;
        heap_push(h, &sz, (heap_item){nd, v});
      }
    }
  }
  int rc = 0;
  for (int32_t v = 0; v < n; ++v) {
    if (d[v] == UINT64_MAX) dist_out[v] = ORACLE_INF;
    else if (d[v] >= ORACLE_INF) { dist_out[v] = ORACLE_INF; rc = 1; }
    else dist_out[v] = (uint32_t)d[v];
  }
  free(d); free(done); free(h);
  return rc;
}

/*
 * Frontier rounds of edge relaxation (the loop that the SSSP kernel of Fig. 1b
 * runs when it is applied repeatedly). Round r takes the frontier F_r (the
 * vertices whose distance dropped in round r-1; F_0 = {source}) and the
 * distances as they stood when round r began; every edge (u,v,w) with u in F_r
 * offers d(u)+w to v, and v enters F_{r+1} when its distance drops. Rounds stop
 * when the frontier is empty. Because every round reads only distances fixed at
 * the end of the previous round, the frontier sets do not depend on the order in
 * which the relaxations of a round are carried out.
 *
 * For each round r: frontier_size[r] = |F_r|, heavy[r] = #{u in F_r : deg(u) >
 * threshold} (the vertices for which the basic-DP kernel launches a child).
 * Arrays must hold max_rounds entries. Returns the number of rounds, or -1 on
 * bad arguments / more than max_rounds rounds / distance overflow.
 * *relaxations = number of edges examined over all rounds.
 */
int64_t oracle_sssp_frontier(int32_t n, const int32_t *off, const int32_t *col, const uint32_t *w, int32_t source,
                             int32_t threshold, uint32_t *dist_out, int64_t max_rounds, int64_t *frontier_size,
                             int64_t *heavy, int64_t *relaxations) {
  if (n < 1 || source < 0 || source >= n) return -1;
  uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint64_t *dprev = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  int32_t *F = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *G = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  uint8_t *in_next = (uint8_t *)calloc((size_t)n, 1);
  if (!d || !dprev || !F || !G || !in_next) {
    free(d); free(dprev); free(F); free(G); free(in_next);
    return -1;
  }
  for (int32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  d[source] = 0;
  int64_t nf = 1, rounds = 0, relax = 0;
  F[0] = source;
  int bad = 0;
  while (nf > 0) {
    if (rounds >= max_rounds) { bad = 1; break; }
    int64_t hv = 0;
    for (int64_t i = 0; i < nf; ++i) if (off[F[i] + 1] - off[F[i]] > threshold) hv++;
    frontier_size[rounds] = nf;
    heavy[rounds] = hv;
    /* distances as they stood when the round began */
    for (int64_t i = 0; i < nf; ++i) dprev[F[i]] = d[F[i]];
    int64_t ng = 0;
    for (int64_t i = 0; i < nf; ++i) {
      int32_t u = F[i];
      for (int64_t e = off[u]; e < off[u + 1]; ++e) {
        int32_t v = col[e];
        uint64_t nd = dprev[u] + (uint64_t)w[e];
        relax++;
        if (nd < d[v]) {
          d[v] = nd;
          if (!in_next[v]) { in_next[v] = 1; G[ng++] = v; }
        }
      }
    }
    for (int64_t i = 0; i < ng; ++i) in_next[G[i]] = 0;
    int32_t *t = F; F = G; G = t;
    nf = ng;
    rounds++;
  }
  for (int32_t v = 0; v < n; ++v) {
    if (d[v] == UINT64_MAX) dist_out[v] = ORACLE_INF;
    else if (d[v] >= ORACLE_INF) { dist_out[v] = ORACLE_INF; bad = 1; }
    else dist_out[v] = (uint32_t)d[v];
  }
  *relaxations = relax;
  free(d); free(dprev); free(F); free(G); free(in_next);
  return bad ? -1 : rounds;
}

/*
 * Near-far frontier rounds: the rounds of oracle_sssp_frontier with the
 * near-far work split of Davidson, Baxter, Garland & Owens ("Work-Efficient
 * Parallel GPU Methods for Single-Source Shortest Paths", IPDPS 2014) put in
 * front of them, and a finer split for heavy vertices.
 *
 * A split distance S, always a multiple of delta, divides the vertices whose
 * distance dropped in a round: those with d < S join the near set, the others
 * the far pile (a set: a vertex is in it at most once). A round relaxes part
 * of the near set, Jacobi-style as in oracle_sssp_frontier (each relaxed
 * vertex offers the distance it had when the round began).
 *
 * Which near vertices a round relaxes: a vertex whose out-degree is at most
 * `threshold` always; a heavy one (out-degree above the threshold) only when
 * its distance is below the sub-split s, a multiple of sub_delta; the other
 * heavy ones stay in the near set for a later round. When no near vertex
 * qualifies, s advances to sub_delta * (floor(hmin / sub_delta) + 1), hmin the
 * smallest distance in the near set (a sub-split advance). sub_delta = 0: no
 * sub-split (every near vertex qualifies).
 *
 * When the near set is empty the split advances:
 *   - far-pile vertices with d < S were relaxed with their current distance
 *     already (they dropped below S, so they went through the near set) and
 *     are dropped;
 *   - dmin = the smallest distance among the others; S becomes
 *     delta * (floor(dmin / delta) + 1), the top of dmin's bucket, and s
 *     becomes sub_delta * (floor(dmin / sub_delta) + 1);
 *   - far-pile vertices with d < S (the new) leave the pile and form the near set.
 * The run ends when the near set and the far pile are both empty. delta = 0
 * means no split (S infinite): with sub_delta = 0 too, exactly the rounds of
 * oracle_sssp_frontier.
 *
 * Per round r: frontier_size[r] = vertices relaxed, heavy[r] = those of them
 * with out-degree above the threshold. *relaxations = edges examined, *splits =
 * split advances, *subsplits = sub-split advances. Returns the number of
 * rounds, or -1 on bad arguments / more than max_rounds rounds / distance
 * overflow.
 */
int64_t oracle_sssp_nearfar(int32_t n, const int32_t *off, const int32_t *col, const uint32_t *w, int32_t source,
                            uint32_t delta, uint32_t sub_delta, int32_t threshold, uint32_t *dist_out,
                            int64_t max_rounds, int64_t *frontier_size, int64_t *heavy, int64_t *relaxations,
                            int64_t *splits, int64_t *subsplits) {
  if (n < 1 || source < 0 || source >= n) return -1;
  uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  uint64_t *dprev = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  int32_t *near = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *act = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *changed = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *far = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  uint8_t *in_near = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *in_changed = (uint8_t *)calloc((size_t)n, 1);
  uint8_t *in_far = (uint8_t *)calloc((size_t)n, 1);
  if (!d || !dprev || !near || !act || !changed || !far || !in_near || !in_changed || !in_far) {
    free(d); free(dprev); free(near); free(act); free(changed); free(far); free(in_near); free(in_changed);
    free(in_far);
    return -1;
  }
  for (int32_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
  d[source] = 0;
  uint64_t S = delta ? (uint64_t)delta : UINT64_MAX;
  uint64_t s = sub_delta ? (uint64_t)sub_delta : UINT64_MAX;
  int64_t nnear = 1, nfar = 0, rounds = 0, relax = 0, nsplit = 0, nsub = 0;
  near[0] = source;
  in_near[source] = 1;
  int bad = 0;
  for (;;) {
    if (nnear == 0) {
      if (nfar == 0) break;
      /* advance the split */
      uint64_t dmin = UINT64_MAX;
      for (int64_t i = 0; i < nfar; ++i)
        if (d[far[i]] >= S && d[far[i]] < dmin) dmin = d[far[i]];
      if (dmin == UINT64_MAX) { /* every far vertex was stale */
        for (int64_t i = 0; i < nfar; ++i) in_far[far[i]] = 0;
        nfar = 0;
        break;
      }
      const uint64_t S_old = S;
      S = (dmin / delta + 1) * (uint64_t)delta;
      if (sub_delta) s = (dmin / sub_delta + 1) * (uint64_t)sub_delta;
      nsplit++;
      int64_t keep = 0;
      for (int64_t i = 0; i < nfar; ++i) {
        int32_t v = far[i];
        if (d[v] < S_old) { in_far[v] = 0; continue; } /* relaxed already */
        if (d[v] < S) {                                 /* the new near set */
          in_far[v] = 0;
          near[nnear++] = v;
          in_near[v] = 1;
          continue;
        }
        far[keep++] = v;
      }
      nfar = keep;
      continue;
    }
    if (rounds >= max_rounds) { bad = 1; break; }
    /* the near vertices this round relaxes */
    int64_t na = 0;
    for (int64_t i = 0; i < nnear; ++i) {
      int32_t v = near[i];
      if (off[v + 1] - off[v] <= threshold || d[v] < s) act[na++] = v;
    }
    if (na == 0) { /* only heavy vertices at or above the sub-split: advance it */
      uint64_t hmin = UINT64_MAX;
      for (int64_t i = 0; i < nnear; ++i) if (d[near[i]] < hmin) hmin = d[near[i]];
      s = (hmin / sub_delta + 1) * (uint64_t)sub_delta;
      nsub++;
      for (int64_t i = 0; i < nnear; ++i) if (d[near[i]] < s) act[na++] = near[i];
    }
    /* the rest stay in the near set */
    int64_t keep = 0;
    for (int64_t i = 0, j = 0; i < nnear; ++i) {
      if (j < na && near[i] == act[j]) { in_near[near[i]] = 0; j++; continue; }
      near[keep++] = near[i];
    }
    nnear = keep;
    int64_t hv = 0;
    for (int64_t i = 0; i < na; ++i) if (off[act[i] + 1] - off[act[i]] > threshold) hv++;
    frontier_size[rounds] = na;
    heavy[rounds] = hv;
    for (int64_t i = 0; i < na; ++i) dprev[act[i]] = d[act[i]];
    int64_t nc = 0;
    for (int64_t i = 0; i < na; ++i) {
      int32_t u = act[i];
      for (int64_t e = off[u]; e < off[u + 1]; ++e) {
        int32_t v = col[e];
        uint64_t nd = dprev[u] + (uint64_t)w[e];
        relax++;
        if (nd < d[v]) {
          d[v] = nd;
          if (!in_changed[v]) { in_changed[v] = 1; changed[nc++] = v; }
        }
      }
    }
    rounds++;
    /* the vertices that dropped: into the near set or the far pile */
    for (int64_t i = 0; i < nc; ++i) {
      int32_t v = changed[i];
      in_changed[v] = 0;
      if (d[v] < S) {
        if (!in_near[v]) { in_near[v] = 1; near[nnear++] = v; }
      } else if (!in_far[v]) {
        in_far[v] = 1;
        far[nfar++] = v;
      }
    }
  }
  for (int32_t v = 0; v < n; ++v) {
    if (d[v] == UINT64_MAX) dist_out[v] = ORACLE_INF;
    else if (d[v] >= ORACLE_INF) { dist_out[v] = ORACLE_INF; bad = 1; }
    else dist_out[v] = (uint32_t)d[v];
  }
  *relaxations = relax;
  if (splits) *splits = nsplit;
  if (subsplits) *subsplits = nsub;
  free(d); free(dprev); free(near); free(act); free(changed); free(far); free(in_near); free(in_changed);
  free(in_far);
  return bad ? -1 : rounds;
}

/* ------------------------------------------------------------------ SpMV */

/*
 * y[i] = sum_k val[k] * x[col[k]] over row i, in double precision, plus
 * absrow[i] = sum_k |val[k] * x[col[k]]| (the scale of row i used by the
 * row-relative error test). Empty rows give 0. Returns 0, -1 on bad arguments.
 */
int oracle_spmv_f64(int32_t nrows, int32_t ncols, const int32_t *off, const int32_t *col, const float *val,
                    const float *x, double *y, double *absrow) {
  if (nrows < 0 || ncols < 0) return -1;
  for (int32_t i = 0; i < nrows; ++i) {
    double s = 0.0, a = 0.0;
    for (int64_t k = off[i]; k < off[i + 1]; ++k) {
      int32_t j = col[k];
      if (j < 0 || j >= ncols) return -1;
      double p = (double)val[k] * (double)x[j];
      s += p;
      a += p < 0 ? -p : p;
    }
    y[i] = s;
    if (absrow) absrow[i] = a;
  }
  return 0;
}

/* ------------------------------------------------------------------ trees */

/*
 * Depth-first post-order with an explicit stack (the recursion of Fig. 1c: a
 * node is finished only after every child's subtree is finished). Checks that
 * the child lists describe a tree rooted at `root` spanning all n nodes: every
 * node reached exactly once. Writes the order in which nodes finish to post[]
 * and each node's depth. Returns 0, or -1 if the input is not such a tree.
 */
static int tree_postorder(int32_t n, const int32_t *coff, const int32_t *cidx, int32_t root, int32_t *post,
                          int32_t *depth) {
  if (n < 1 || root < 0 || root >= n) return -1;
  if (coff[0] != 0 || coff[n] != n - 1) return -1;
  uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
  int32_t *stack = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t *next = (int64_t *)malloc((size_t)n * sizeof(int64_t)); /* next child slot to visit */
  if (!seen || !stack || !next) { free(seen); free(stack); free(next); return -1; }
  int64_t sp = 0, np = 0;
  int rc = 0;
  stack[sp++] = root;
  seen[root] = 1;
  depth[root] = 0;
  next[root] = coff[root];
  while (sp > 0) {
    int32_t v = stack[sp - 1];
    if (next[v] < coff[v + 1]) {
      int32_t c = cidx[next[v]++];
      if (c < 0 || c >= n || seen[c]) { rc = -1; break; }
      seen[c] = 1;
      depth[c] = depth[v] + 1;
      next[c] = coff[c];
      stack[sp++] = c;
    } else {
      post[np++] = v;
      sp--;
    }
  }
  if (rc == 0 && np != n) rc = -1;
  free(seen); free(stack); free(next);
  return rc;
}

/* desc(v) = sum over children c of (1 + desc(c)); leaves 0. Returns 0 / -1. */
int oracle_tree_descendants(int32_t n, const int32_t *coff, const int32_t *cidx, int32_t root, uint32_t *desc) {
  int32_t *post = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t *depth = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int rc = tree_postorder(n, coff, cidx, root, post, depth);
  if (rc == 0) {
    for (int32_t i = 0; i < n; ++i) {
      int32_t v = post[i];
      uint64_t s = 0;
      for (int64_t k = coff[v]; k < coff[v + 1]; ++k) s += 1 + (uint64_t)desc[cidx[k]];
      desc[v] = (uint32_t)s;
    }
  }
  free(post); free(depth);
  return rc;
}

/* height(leaf) = 0, height(v) = 1 + max over children of height(c). Returns 0 / -1. */
int oracle_tree_height(int32_t n, const int32_t *coff, const int32_t *cidx, int32_t root, int32_t *height) {
  int32_t *post = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t *depth = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int rc = tree_postorder(n, coff, cidx, root, post, depth);
  if (rc == 0) {
    for (int32_t i = 0; i < n; ++i) {
      int32_t v = post[i];
      int32_t h = 0;
      for (int64_t k = coff[v]; k < coff[v + 1]; ++k) {
        int32_t hc = 1 + height[cidx[k]];
        if (hc > h) h = hc;
      }
      height[v] = h;
    }
  }
  free(post); free(depth);
  return rc;
}

/*
 * Per-depth structure of the recursion. For depth L in [0, max_levels):
 * nodes[L] = #nodes at depth L, internal[L] = #nodes at depth L with at least
 * one child, edges[L] = #child edges leaving depth L, heavy[L] = #nodes at depth
 * L whose child count exceeds threshold. Returns the number of depths (max
 * depth + 1), or -1 on a malformed tree or more than max_levels depths.
 */
int32_t oracle_tree_levels(int32_t n, const int32_t *coff, const int32_t *cidx, int32_t root, int32_t threshold,
                           int32_t max_levels, int64_t *nodes, int64_t *internal, int64_t *edges, int64_t *heavy) {
  int32_t *post = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t *depth = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int rc = tree_postorder(n, coff, cidx, root, post, depth);
  int32_t levels = -1;
  if (rc == 0) {
    levels = 0;
    for (int32_t v = 0; v < n; ++v) if (depth[v] + 1 > levels) levels = depth[v] + 1;
    if (levels > max_levels) {
      levels = -1;
    } else {
      for (int32_t L = 0; L < levels; ++L) nodes[L] = internal[L] = edges[L] = heavy[L] = 0;
      for (int32_t v = 0; v < n; ++v) {
        int64_t k = coff[v + 1] - coff[v];
        int32_t L = depth[v];
        nodes[L]++;
        if (k > 0) internal[L]++;
        edges[L] += k;
        if (k > threshold) heavy[L]++;
      }
    }
  }
  free(post); free(depth);
  return levels;
}

/* ------------------------------------------------------------------ launch counts */

/*
 * Child-kernel launches of one parent grid under each consolidation granularity
 * (Sec. IV.B). The parent grid has `blocks` blocks of `threads` threads; global
 * thread g = b*threads + t takes items g, g + G, g + 2G, ... (G = blocks*threads)
 * and buffers the items whose flag is set. Warps are groups of 32 consecutive
 * threads of one block.
 *   out[0] basic-DP : one launch per buffered item
 *   out[1] flat     : no launches
 *   out[2] warp     : one launch per warp that buffered at least one item
 *   out[3] block    : one launch per block that buffered at least one item
 *   out[4] grid     : one launch if any item was buffered
 * Returns 0, -1 on bad arguments.
 */
int oracle_consolidation_launches(int64_t nitems, const uint8_t *flag, int32_t blocks, int32_t threads,
                                  int64_t out[5]) {
  if (nitems < 0 || blocks < 1 || threads < 1) return -1;
  int64_t G = (int64_t)blocks * threads;
  int32_t warps_per_block = (threads + 31) / 32;
  uint8_t *warp_hit = (uint8_t *)calloc((size_t)blocks * warps_per_block, 1);
  uint8_t *block_hit = (uint8_t *)calloc((size_t)blocks, 1);
  if (!warp_hit || !block_hit) { free(warp_hit); free(block_hit); return -1; }
  int64_t basic = 0;
  for (int64_t i = 0; i < nitems; ++i) {
    if (!flag[i]) continue;
    basic++;
    int64_t g = i % G;
    int32_t b = (int32_t)(g / threads), t = (int32_t)(g % threads);
    warp_hit[(int64_t)b * warps_per_block + t / 32] = 1;
    block_hit[b] = 1;
  }
  int64_t nw = 0, nb = 0;
  for (int64_t k = 0; k < (int64_t)blocks * warps_per_block; ++k) nw += warp_hit[k];
  for (int32_t b = 0; b < blocks; ++b) nb += block_hit[b];
  out[0] = basic;
  out[1] = 0;
  out[2] = nw;
  out[3] = nb;
  out[4] = basic > 0 ? 1 : 0;
  free(warp_hit); free(block_hit);
  return 0;
}

/* ------------------------------------------------------------------ PageRank */

/*
 * PageRank, the PR benchmark of Sec. V (the paper names the application and
 * its irregular per-vertex loop; the definition is the usual one, with the
 * readings below). Graph given by its OUT-edge CSR: off[n+1], col[m] in [0,n);
 * duplicate edges and self-loops count with their multiplicity.
 *   rank_0(v)     = 1/n
 *   D_t           = sum of rank_t(u) over vertices u without out-edges
 *   rank_{t+1}(v) = (1-d)/n + d * ( D_t/n + sum over edges (u,v) of rank_t(u)/outdeg(u) )
 * for t = 0 .. iters-1, in double precision, each vertex's rank pushed along
 * its out-edges (the GPU path pulls over in-edges instead). Writes rank_iters.
 * Returns 0, -1 on bad arguments or memory.
 */
int oracle_pagerank(int32_t n, const int32_t *off, const int32_t *col, double d, int32_t iters, double *rank) {
  if (n < 1 || iters < 0 || !(d >= 0.0 && d <= 1.0)) return -1;
  if (off[0] != 0) return -1;
  for (int32_t u = 0; u < n; ++u)
    if (off[u + 1] < off[u]) return -1;
  for (int64_t k = 0; k < off[n]; ++k)
    if (col[k] < 0 || col[k] >= n) return -1;
  double *next = (double *)malloc(sizeof(double) * (size_t)n);
  if (!next) return -1;
  for (int32_t v = 0; v < n; ++v) rank[v] = 1.0 / (double)n;
  for (int32_t t = 0; t < iters; ++t) {
    double dangling = 0.0;
    for (int32_t u = 0; u < n; ++u)
      if (off[u + 1] == off[u]) dangling += rank[u];
    for (int32_t v = 0; v < n; ++v) next[v] = 0.0;
    for (int32_t u = 0; u < n; ++u) {
      int64_t deg = (int64_t)off[u + 1] - off[u];
      if (deg == 0) continue;
      double share = rank[u] / (double)deg;
      for (int64_t k = off[u]; k < off[u + 1]; ++k) next[col[k]] += share;
    }
    for (int32_t v = 0; v < n; ++v) rank[v] = (1.0 - d) / (double)n + d * (dangling / (double)n + next[v]);
  }
  free(next);
  return 0;
}

/* ------------------------------------------------------------------ BFS */

/*
 * Breadth-first levels, the result of the recursive BFS benchmark (BFS-Rec,
 * Sec. V): level[v] = fewest edges on a path from `source` to v, 0xFFFFFFFF
 * when v is unreachable. Textbook FIFO-queue BFS over the out-edge CSR;
 * duplicate edges and self-loops are allowed. Returns the number of distinct
 * levels (the depth of the BFS tree plus one), -1 on bad arguments or memory.
 */
int32_t oracle_bfs(int32_t n, const int32_t *off, const int32_t *col, int32_t source, uint32_t *level) {
  if (n < 1 || source < 0 || source >= n || off[0] != 0) return -1;
  for (int32_t u = 0; u < n; ++u)
    if (off[u + 1] < off[u]) return -1;
  for (int64_t k = 0; k < off[n]; ++k)
    if (col[k] < 0 || col[k] >= n) return -1;
  int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!queue) return -1;
  for (int32_t v = 0; v < n; ++v) level[v] = ORACLE_INF;
  int64_t head = 0, tail = 0;
  level[source] = 0;
  queue[tail++] = source;
  uint32_t deepest = 0;
  while (head < tail) {
    const int32_t u = queue[head++];
    for (int64_t k = off[u]; k < off[u + 1]; ++k) {
      const int32_t v = col[k];
      if (level[v] == ORACLE_INF) {
        level[v] = level[u] + 1;
        if (level[v] > deepest) deepest = level[v];
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return (int32_t)deepest + 1;
}

/* ------------------------------------------------------------------ graph colouring */

/* u outranks v: higher priority, ties broken by the larger vertex id. */
static int outranks(const uint32_t *prio, int32_t u, int32_t v) {
  return prio[u] > prio[v] || (prio[u] == prio[v] && u > v);
}

/*
 * Graph colouring, the GC benchmark of Sec. V (the paper names the benchmark;
 * the algorithm read here is the independent-set rounds of Jones-Plassmann
 * with the priorities given as input, the colour being the round). Symmetric CSR off[n+1], col[m] (self-loops ignored, duplicates
 * harmless). Rounds r = 1, 2, ...: a vertex still uncoloured when round r
 * begins takes colour r unless a neighbour also uncoloured when the round began
 * outranks it. Writes color[n] (>= 1), and per round (arrays of capacity
 * `cap`, may be NULL) the number of uncoloured vertices and how many of them
 * have more than `threshold` neighbours (the large work items). Returns the
 * number of rounds (the number of colours), -1 on bad arguments or memory, -2
 * when more than `cap` rounds were needed.
 */
int32_t oracle_color_jp(int32_t n, const int32_t *off, const int32_t *col, const uint32_t *prio, int32_t threshold,
                        int32_t *color, int64_t cap, int64_t *active_per_round, int64_t *heavy_per_round) {
  if (n < 1 || off[0] != 0 || threshold < 0) return -1;
  for (int32_t u = 0; u < n; ++u)
    if (off[u + 1] < off[u]) return -1;
  for (int64_t k = 0; k < off[n]; ++k)
    if (col[k] < 0 || col[k] >= n) return -1;
  int32_t *at_start = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!at_start) return -1;
  for (int32_t v = 0; v < n; ++v) color[v] = 0;
  int32_t r = 0;
  int64_t left = n;
  while (left > 0) {
    ++r;
    int64_t active = 0, heavy = 0;
    for (int32_t v = 0; v < n; ++v) {
      at_start[v] = color[v];
      if (color[v] == 0) {
        active++;
        if (off[v + 1] - off[v] > threshold) heavy++;
      }
    }
    if (r <= cap) {
      if (active_per_round) active_per_round[r - 1] = active;
      if (heavy_per_round) heavy_per_round[r - 1] = heavy;
    }
    for (int32_t v = 0; v < n; ++v) {
      if (at_start[v] != 0) continue;
      int blocked = 0;
      for (int64_t k = off[v]; k < off[v + 1] && !blocked; ++k) {
        const int32_t u = col[k];
        if (u != v && at_start[u] == 0 && outranks(prio, u, v)) blocked = 1;
      }
      if (!blocked) {
        color[v] = r;
        left--;
      }
    }
  }
  free(at_start);
  return r <= cap || cap <= 0 ? r : -2;
}
