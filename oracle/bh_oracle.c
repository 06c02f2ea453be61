/*
 * CPU oracle for the Barnes-Hut potential on an octree AMR mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library: it is a plain, slow, separately written statement of what the
 * method computes, in FP64.
 *
 * What it computes (paper = Lukat & Banerjee, "A GPU accelerated Barnes-Hut
 * tree code for FLASH4"):
 *   - The octree (Sec. 2; Sec. 3.2.2): one cube holds the whole box and is
 *     split recursively into 8 sub-cubes until every sub-cube holds one item.
 *     The items are the AMR cells (footnote in Sec. 2: cells are the
 *     "particles"); because the leaf blocks tile the box, the recursion meets
 *     every leaf block as a node and continues inside it down to single cells
 *     (the FLASH tree solver's "extension of the AMR mesh tree down to the
 *     individual cells", Sec. 1).  Children are kept in octant order
 *     o = ox + 2*oy + 4*oz.
 *   - Node moments (Sec. 3.2.3, Eq. 5): M = sum of the children's masses,
 *     R = (1/M) sum m_i r_i over the children in octant order, and delta =
 *     |R - geometric centre| (Sec. 2, Fig. opening_angles).  Leaf mass is
 *     rho * cell volume, leaf position the cell centre.
 *   - The walk (Sec. 2, Eqs. 3-4; Sec. 3.3): from the root, a node is
 *     accepted for target t when d > l/theta + delta (d = |r_t - R|, l = node
 *     side) and contributes -G M / d; otherwise its 8 children are visited.
 *     A leaf cell other than t always contributes -G m / d.
 *   - Direct sum (Eq. 2) without the printed factor 1/2 (that factor belongs
 *     to the total-energy sum, not to the potential at one cell).
 *   - Paper mode (Sec. 3.3): 32 neighbouring cells (a 4x4x2 brick of a block)
 *     walk together and a node is accepted only if all 32 accept it
 *     (warp vote all()).
 *   - Optional quadrupole term (not in the paper; the textbook next term of
 *     the multipole expansion about the centre of mass): each node carries
 *     its traceless quadrupole Q = sum over its cells of m (3 x x^T - |x|^2 I),
 *     x = cell centre - R, computed here straight from that definition, and an
 *     accepted node contributes -G (M/d + (1/2) d^T Q d / d^5), d = r_t - R.
 *     The opening test is unchanged; cells carry no quadrupole.
 *   - Periodic boundaries (App. A): the Ewald field replaces 1/d in every
 *     term, tabulated and interpolated quadratically; see the section
 *     "periodic boundaries" below.
 *   - Optional learned correction (not in the paper): each accepted node's
 *     term M/d is multiplied by (1 + s^2 y), y = MLP(x), where s = l/d and x
 *     holds ten features of the (target, node) pair (see pair_features); the
 *     MLP is 10 -> 64 -> 64 -> 1 with tanh-form GELU activations, evaluated
 *     here in FP64 with the weights it is given.  The training residual of a
 *     pair is eps = (sum over the node's cells of m / |r_t - r_c|)/(M/d) - 1,
 *     the node's exact contribution against its monopole.
 *
 * Readings where the paper is silent (each also stated in the design notes):
 *   - Positions are taken in box units u = (x - lo)/L, so Phi = -(G/L) sum M/|du|.
 *   - The acceptance test is evaluated in IEEE binary32 with this fixed order
 *     of operations, so that any implementation that evaluates it in binary32
 *     reaches the same decision (the interaction sum itself stays FP64 here):
 *       inv = (float)(1/theta)          l = (float)2^-level
 *       s   = fl(fl(l*inv) + (float)delta)
 *       s2  = fl(s*s)
 *       P   = (float)R,  t = (float)u_t (exact: cell centres are dyadic)
 *       dx  = fl(t.x - P.x), ...
 *       d2  = fma(dx,dx, fma(dz,dz, fl(dy*dy)))
 *       accept  <=>  d2 > s2
 *     This file is compiled with -ffp-contract=off so that every fl() above
 *     is a single rounding.
 *   - A node of zero mass has R = its geometric centre (delta = 0).
 *   - Sums over accepted terms use Neumaier's compensated summation in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_GEOMETRY 2
#define OR_ERR_OOM 3

#define MAX_BLOCK_LEVEL 18

typedef struct {
  int level;          /* 0 = the whole box */
  int64_t ijk[3];     /* integer position of the cube at its level */
  int child[8];       /* node index per octant, or -1 for a leaf */
  int64_t cell;       /* caller cell index b*512 + cz*64 + cy*8 + cx (leaves) */
  int parent;
  double M;           /* mass */
  double R[3];        /* centre of mass, box units */
  double delta;       /* |R - geometric centre|, box units */
  double Q[6];        /* quadrupole about R: xx, yy, zz, xy, xz, yz (box units) */
} onode;

typedef struct {
  int nblocks;
  double lo[3], L;
  int64_t nnodes, cap;
  onode *node;
  int64_t *leaf_of_cell; /* caller cell index -> node index */
  /* build scratch */
  const int *blevel;
  const int *bijk;
  const double *rho;
  uint64_t *bkey;      /* corner keys of blocks, sorted */
  int *border;         /* block index, in key order */
  int used_blocks;
  int err;
  int have_quad;
} otree;

/* ---------------------------------------------------------------- keys -- */
static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}
/* Morton key of the lower corner of cube (level, i, j, k) on the level-21
 * lattice.  Octant order o = ox + 2 oy + 4 oz gives x the lowest bit. */
static uint64_t corner_key(int level, int64_t i, int64_t j, int64_t k) {
  int sh = 21 - level;
  return spread3((uint64_t)i << sh) | (spread3((uint64_t)j << sh) << 1) |
         (spread3((uint64_t)k << sh) << 2);
}

static otree *g_sort_tree;
static int cmp_block(const void *a, const void *b) {
  int x = *(const int *)a, y = *(const int *)b;
  uint64_t kx = g_sort_tree->bkey[x], ky = g_sort_tree->bkey[y];
  return kx < ky ? -1 : kx > ky ? 1 : (x - y);
}

/* First position in key order whose key is >= k. */
static int lower_bound_key(const otree *t, const uint64_t *sorted, uint64_t k) {
  int a = 0, b = t->nblocks;
  while (a < b) {
    int m = (a + b) / 2;
    if (sorted[m] < k) a = m + 1; else b = m;
  }
  return a;
}

/* ---------------------------------------------------------------- build -- */
static int new_node(otree *t, int level, int64_t i, int64_t j, int64_t k, int parent) {
  if (t->nnodes == t->cap) {
    int64_t nc = t->cap ? 2 * t->cap : 1024;
    onode *p = (onode *)realloc(t->node, (size_t)nc * sizeof(onode));
    if (!p) { t->err = OR_ERR_OOM; return -1; }
    t->node = p;
    t->cap = nc;
  }
  int id = (int)t->nnodes++;
  onode *n = &t->node[id];
  memset(n, 0, sizeof(*n));
  n->level = level;
  n->ijk[0] = i; n->ijk[1] = j; n->ijk[2] = k;
  for (int o = 0; o < 8; ++o) n->child[o] = -1;
  n->cell = -1;
  n->parent = parent;
  return id;
}

/* Subtree of the cube (level, i,j,k) that lies inside block b (depth d in
 * the block: 0 = the block itself, 3 = a single cell). */
static int make_in_block(otree *t, int b, int d, int level, int64_t i, int64_t j,
                         int64_t k, int parent) {
  int id = new_node(t, level, i, j, k, parent);
  if (id < 0) return -1;
  if (d == 3) {
    int64_t cx = i - 8 * (int64_t)t->bijk[3 * b + 0];
    int64_t cy = j - 8 * (int64_t)t->bijk[3 * b + 1];
    int64_t cz = k - 8 * (int64_t)t->bijk[3 * b + 2];
    t->node[id].cell = (int64_t)b * 512 + cz * 64 + cy * 8 + cx;
    return id;
  }
  for (int o = 0; o < 8; ++o) {
    int c = make_in_block(t, b, d + 1, level + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1),
                          2 * k + ((o >> 2) & 1), id);
    if (c < 0) return -1;
    t->node[id].child[o] = c;
  }
  return id;
}

static const uint64_t *g_sorted_keys;

/* Cube (level, i,j,k): it is either exactly one leaf block, or it is covered
 * by finer blocks and split into 8 children. */
static int make_cube(otree *t, int level, int64_t i, int64_t j, int64_t k, int parent) {
  uint64_t k0 = corner_key(level, i, j, k);
  uint64_t span = 1ull << (3 * (21 - level)); /* level 0: 2^63, fits */
  int a = lower_bound_key(t, g_sorted_keys, k0);
  int e = (k0 + span == 0) ? t->nblocks : lower_bound_key(t, g_sorted_keys, k0 + span);
  if (level == 0) e = t->nblocks;
  if (a >= e) { t->err = OR_ERR_GEOMETRY; return -1; } /* gap */
  int b0 = t->border[a];
  if (g_sorted_keys[a] == k0 && t->blevel[b0] <= level) {
    /* a block starts here at this level or coarser */
    if (t->blevel[b0] != level || e - a != 1) { t->err = OR_ERR_GEOMETRY; return -1; }
    t->used_blocks++;
    return make_in_block(t, b0, 0, level, i, j, k, parent);
  }
  if (level >= MAX_BLOCK_LEVEL) { t->err = OR_ERR_GEOMETRY; return -1; }
  int id = new_node(t, level, i, j, k, parent);
  if (id < 0) return -1;
  for (int o = 0; o < 8; ++o) {
    int c = make_cube(t, level + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1),
                      2 * k + ((o >> 2) & 1), id);
    if (c < 0) return -1;
    t->node[id].child[o] = c;
  }
  return id;
}

/* Moments, Eq. 5.  Node indices are in pre-order (children after parents),
 * so one pass over decreasing index sees every child before its parent. */
static void compute_moments(otree *t) {
  for (int64_t id = t->nnodes - 1; id >= 0; --id) {
    onode *n = &t->node[id];
    double side = ldexp(1.0, -n->level);                /* box units */
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = ((double)n->ijk[a] + 0.5) * side;
    if (n->child[0] < 0) {
      /* leaf: m = rho * cell volume (physical), position = cell centre */
      int64_t cell = n->cell;
      double h = t->L * ldexp(1.0, -n->level);
      double vol = h * h * h;
      n->M = t->rho[cell] * vol;
      for (int a = 0; a < 3; ++a) n->R[a] = c[a];
      n->delta = 0.0;
      continue;
    }
    double M = 0.0, S[3] = {0.0, 0.0, 0.0};
    for (int o = 0; o < 8; ++o) {
      const onode *ch = &t->node[n->child[o]];
      M = M + ch->M;
      for (int a = 0; a < 3; ++a) S[a] = S[a] + ch->M * ch->R[a];
    }
    n->M = M;
    if (M > 0.0) {
      for (int a = 0; a < 3; ++a) n->R[a] = S[a] / M;
    } else {
      for (int a = 0; a < 3; ++a) n->R[a] = c[a];
    }
    double o0 = n->R[0] - c[0], o1 = n->R[1] - c[1], o2 = n->R[2] - c[2];
    n->delta = sqrt((o0 * o0 + o1 * o1) + o2 * o2);
  }
}

int or_build(int nblocks, const int *level, const int *ijk, const double *density,
             const double *lo, double L, void **out) {
  *out = NULL;
  if (nblocks <= 0 || !level || !ijk || !density || !lo || !(L > 0.0)) return OR_ERR_ARG;
  for (int b = 0; b < nblocks; ++b) {
    if (level[b] < 0 || level[b] > MAX_BLOCK_LEVEL) return OR_ERR_GEOMETRY;
    int64_t n = (int64_t)1 << level[b];
    for (int a = 0; a < 3; ++a)
      if (ijk[3 * b + a] < 0 || ijk[3 * b + a] >= n) return OR_ERR_GEOMETRY;
  }
  for (int64_t c = 0; c < (int64_t)nblocks * 512; ++c)
    if (!(density[c] >= 0.0) || !isfinite(density[c])) return OR_ERR_ARG;
  otree *t = (otree *)calloc(1, sizeof(otree));
  if (!t) return OR_ERR_OOM;
  t->nblocks = nblocks;
  for (int a = 0; a < 3; ++a) t->lo[a] = lo[a];
  t->L = L;
  t->blevel = level;
  t->bijk = ijk;
  t->rho = density;
  t->bkey = (uint64_t *)malloc(sizeof(uint64_t) * nblocks);
  t->border = (int *)malloc(sizeof(int) * nblocks);
  uint64_t *sk = (uint64_t *)malloc(sizeof(uint64_t) * nblocks);
  if (!t->bkey || !t->border || !sk) { free(sk); free(t->bkey); free(t->border); free(t); return OR_ERR_OOM; }
  for (int b = 0; b < nblocks; ++b) {
    t->bkey[b] = corner_key(level[b], ijk[3 * b], ijk[3 * b + 1], ijk[3 * b + 2]);
    t->border[b] = b;
  }
  g_sort_tree = t;
  qsort(t->border, nblocks, sizeof(int), cmp_block);
  for (int p = 0; p < nblocks; ++p) sk[p] = t->bkey[t->border[p]];
  g_sorted_keys = sk;
  t->err = OR_OK;
  make_cube(t, 0, 0, 0, 0, -1);
  if (t->err == OR_OK && t->used_blocks != nblocks) t->err = OR_ERR_GEOMETRY;
  free(sk);
  g_sorted_keys = NULL;
  int err = t->err;
  if (err == OR_OK) {
    t->leaf_of_cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)nblocks * 512);
    if (!t->leaf_of_cell) err = OR_ERR_OOM;
  }
  if (err != OR_OK) {
    free(t->node); free(t->bkey); free(t->border); free(t->leaf_of_cell); free(t);
    return err;
  }
  for (int64_t id = 0; id < t->nnodes; ++id)
    if (t->node[id].child[0] < 0) t->leaf_of_cell[t->node[id].cell] = id;
  compute_moments(t);
  t->rho = NULL; t->blevel = NULL; t->bijk = NULL;
  *out = t;
  return OR_OK;
}

void or_free(void *p) {
  otree *t = (otree *)p;
  if (!t) return;
  free(t->node); free(t->bkey); free(t->border); free(t->leaf_of_cell); free(t);
}

int64_t or_num_nodes(const void *p) { return ((const otree *)p)->nnodes; }

/* Node table in pre-order: level, ijk[3], is_leaf, cell, M, R[3], delta,
 * parent.  Any output pointer may be NULL. */
int or_export(const void *p, int32_t *level, int64_t *ijk, int32_t *is_leaf, int64_t *cell,
              double *M, double *R, double *delta, int32_t *parent) {
  const otree *t = (const otree *)p;
  for (int64_t id = 0; id < t->nnodes; ++id) {
    const onode *n = &t->node[id];
    if (level) level[id] = n->level;
    if (ijk) for (int a = 0; a < 3; ++a) ijk[3 * id + a] = n->ijk[a];
    if (is_leaf) is_leaf[id] = n->child[0] < 0;
    if (cell) cell[id] = n->cell;
    if (M) M[id] = n->M;
    if (R) for (int a = 0; a < 3; ++a) R[3 * id + a] = n->R[a];
    if (delta) delta[id] = n->delta;
    if (parent) parent[id] = n->parent;
  }
  return OR_OK;
}

/* Quadrupole of every internal node, from its definition: a sum over the
 * cells of its subtree (a contiguous pre-order range).  Computed on demand. */
int or_quadrupoles(void *p) {
  otree *t = (otree *)p;
  if (t->have_quad) return OR_OK;
  int64_t *end = (int64_t *)malloc(sizeof(int64_t) * (size_t)t->nnodes);
  if (!end) return OR_ERR_OOM;
  for (int64_t id = 0; id < t->nnodes; ++id) end[id] = id + 1;
  for (int64_t id = t->nnodes - 1; id > 0; --id) {
    int64_t par = t->node[id].parent;
    if (end[id] > end[par]) end[par] = end[id];
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (int64_t id = 0; id < t->nnodes; ++id) {
    onode *n = &t->node[id];
    for (int a = 0; a < 6; ++a) n->Q[a] = 0.0;
    if (n->child[0] < 0) continue;
    for (int64_t k = id + 1; k < end[id]; ++k) {
      const onode *c = &t->node[k];
      if (c->child[0] >= 0) continue;
      double x = c->R[0] - n->R[0], y = c->R[1] - n->R[1], z = c->R[2] - n->R[2];
      double r2 = x * x + y * y + z * z;
      n->Q[0] += c->M * (3.0 * x * x - r2);
      n->Q[1] += c->M * (3.0 * y * y - r2);
      n->Q[2] += c->M * (3.0 * z * z - r2);
      n->Q[3] += c->M * (3.0 * x * y);
      n->Q[4] += c->M * (3.0 * x * z);
      n->Q[5] += c->M * (3.0 * y * z);
    }
  }
  free(end);
  t->have_quad = 1;
  return OR_OK;
}

int or_export_quad(const void *p, double *Q) {
  const otree *t = (const otree *)p;
  if (!t->have_quad) return OR_ERR_ARG;
  for (int64_t id = 0; id < t->nnodes; ++id)
    for (int a = 0; a < 6; ++a) Q[6 * id + a] = t->node[id].Q[a];
  return OR_OK;
}

/* ------------------------------------------------------------ the walk -- */
typedef struct { double s, c; } neumaier;
static void nm_add(neumaier *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nm_value(const neumaier *a) { return a->s + a->c; }

/* The binary32 acceptance test of Eq. 4 (rounding spelled out in the header). */
static int accept_f32(const onode *n, const float t[3], float inv_theta) {
  float l = (float)ldexp(1.0, -n->level);
  float s = l * inv_theta;
  s = s + (float)n->delta;
  float s2 = s * s;
  float dx = t[0] - (float)n->R[0];
  float dy = t[1] - (float)n->R[1];
  float dz = t[2] - (float)n->R[2];
  float d2 = fmaf(dx, dx, fmaf(dz, dz, dy * dy));
  return d2 > s2;
}

static double dist64(const double a[3], const double b[3]) {
  double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
  return sqrt((x * x + y * y) + z * z);
}

/* M/d of an accepted node, plus (1/2) d^T Q d / d^5 with the quadrupole. */
static double node_term(const onode *n, const double tu[3], int quad) {
  double d = dist64(tu, n->R);
  if (!quad) return n->M / d;
  double x = tu[0] - n->R[0], y = tu[1] - n->R[1], z = tu[2] - n->R[2];
  double q = n->Q[0] * x * x + n->Q[1] * y * y + n->Q[2] * z * z +
             2.0 * (n->Q[3] * x * y + n->Q[4] * x * z + n->Q[5] * y * z);
  double d2 = d * d;
  return n->M / d + 0.5 * q / (d2 * d2 * d);
}

typedef struct {
  const otree *t;
  int64_t self;
  float tf[3];
  double tu[3];
  float inv_theta;
  int quad;
  neumaier sum;
  int64_t n_int, n_test;
  int64_t *list; int64_t list_n, list_cap;   /* optional accepted-set record */
} walk_state;

static void record(walk_state *w, int64_t id) {
  if (w->list && w->list_n < w->list_cap) w->list[w->list_n] = id;
  w->list_n++;
}

static void walk_node(walk_state *w, int64_t id) {
  const onode *n = &w->t->node[id];
  if (n->child[0] < 0) {                      /* a leaf cell */
    if (id != w->self) {
      nm_add(&w->sum, n->M / dist64(w->tu, n->R));
      w->n_int++;
      record(w, id);
    }
    return;
  }
  w->n_test++;
  if (accept_f32(n, w->tf, w->inv_theta)) {   /* Eq. 4: far enough */
    nm_add(&w->sum, node_term(n, w->tu, w->quad));
    w->n_int++;
    record(w, id);
    return;
  }
  for (int o = 0; o < 8; ++o) walk_node(w, n->child[o]);   /* opened */
}

static void target_position(const otree *t, int64_t leaf, double tu[3], float tf[3]) {
  const onode *n = &t->node[leaf];
  double side = ldexp(1.0, -n->level);
  for (int a = 0; a < 3; ++a) {
    tu[a] = ((double)n->ijk[a] + 0.5) * side;
    tf[a] = (float)tu[a];
  }
}

static int check_theta(double theta) { return theta > 0.0 && theta <= 1.0; }

/* Per-cell walk for the given caller cell indices. */
int or_walk(const void *p, double theta, double G, int quad, int64_t ntargets,
            const int64_t *targets, double *phi, int64_t *n_int, int64_t *n_test, int nthreads) {
  const otree *t = (const otree *)p;
  if (!check_theta(theta) || !isfinite(G)) return OR_ERR_ARG;
  if (quad && !t->have_quad) return OR_ERR_ARG;
  int64_t ncell = (int64_t)t->nblocks * 512;
  for (int64_t q = 0; q < ntargets; ++q)
    if (targets[q] < 0 || targets[q] >= ncell) return OR_ERR_ARG;
  float inv_theta = (float)(1.0 / theta);
  double scale = -G / t->L;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
  for (int64_t q = 0; q < ntargets; ++q) {
    walk_state w;
    memset(&w, 0, sizeof(w));
    w.t = t;
    w.self = t->leaf_of_cell[targets[q]];
    w.inv_theta = inv_theta;
    w.quad = quad;
    target_position(t, w.self, w.tu, w.tf);
    walk_node(&w, 0);
    phi[q] = scale * nm_value(&w.sum);
    if (n_int) n_int[q] = w.n_int;
    if (n_test) n_test[q] = w.n_test;
  }
  return OR_OK;
}

/* Accepted set of one target: node indices (pre-order) of every accepted
 * internal node and every leaf it interacts with.  Returns the count (the
 * list holds the first `cap` of them), or -1 on bad arguments. */
int64_t or_walk_list(const void *p, double theta, int64_t target, int64_t *list, int64_t cap) {
  const otree *t = (const otree *)p;
  if (!check_theta(theta) || target < 0 || target >= (int64_t)t->nblocks * 512) return -1;
  walk_state w;
  memset(&w, 0, sizeof(w));
  w.t = t;
  w.self = t->leaf_of_cell[target];
  w.inv_theta = (float)(1.0 / theta);
  target_position(t, w.self, w.tu, w.tf);
  w.list = list;
  w.list_cap = cap;
  walk_node(&w, 0);
  return w.list_n;
}

/* ------------------------------------------------------ paper mode walk -- */
/* A brick is 32 neighbouring cells of one block: local Morton indices
 * 32q .. 32q+31 (a 4x4x2 set).  All 32 walk together; a node is accepted
 * only when every one of them accepts it (Sec. 3.3, all() vote). */
typedef struct {
  const otree *t;
  int64_t self[32];
  float tf[32][3];
  double tu[32][3];
  float inv_theta;
  int quad;
  neumaier sum[32];
  int64_t n_int[32], n_test[32];
} brick_state;

static void walk_brick(brick_state *w, int64_t id) {
  const onode *n = &w->t->node[id];
  if (n->child[0] < 0) {
    for (int l = 0; l < 32; ++l) {
      if (id == w->self[l]) continue;
      nm_add(&w->sum[l], n->M / dist64(w->tu[l], n->R));
      w->n_int[l]++;
    }
    return;
  }
  int all = 1;
  for (int l = 0; l < 32; ++l) {
    w->n_test[l]++;
    if (!accept_f32(n, w->tf[l], w->inv_theta)) all = 0;
  }
  if (all) {
    for (int l = 0; l < 32; ++l) {
      nm_add(&w->sum[l], node_term(n, w->tu[l], w->quad));
      w->n_int[l]++;
    }
    return;
  }
  for (int o = 0; o < 8; ++o) walk_brick(w, n->child[o]);
}

static int64_t local_morton_to_cell(int64_t b, int m) {
  int cx = 0, cy = 0, cz = 0;
  for (int bit = 0; bit < 3; ++bit) {
    cx |= ((m >> (3 * bit)) & 1) << bit;
    cy |= ((m >> (3 * bit + 1)) & 1) << bit;
    cz |= ((m >> (3 * bit + 2)) & 1) << bit;
  }
  return b * 512 + cz * 64 + cy * 8 + cx;
}

/* bricks[q] = caller block index * 16 + brick number (0..15); phi, n_int and
 * n_test get 32 entries per brick in local Morton order of the cells. */
int or_walk_vote(const void *p, double theta, double G, int quad, int64_t nbricks,
                 const int64_t *bricks, double *phi, int64_t *n_int, int64_t *n_test,
                 int nthreads) {
  const otree *t = (const otree *)p;
  if (!check_theta(theta) || !isfinite(G)) return OR_ERR_ARG;
  if (quad && !t->have_quad) return OR_ERR_ARG;
  for (int64_t q = 0; q < nbricks; ++q)
    if (bricks[q] < 0 || bricks[q] >= (int64_t)t->nblocks * 16) return OR_ERR_ARG;
  float inv_theta = (float)(1.0 / theta);
  double scale = -G / t->L;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t q = 0; q < nbricks; ++q) {
    brick_state *w = (brick_state *)calloc(1, sizeof(brick_state));
    w->t = t;
    w->inv_theta = inv_theta;
    w->quad = quad;
    int64_t b = bricks[q] / 16;
    int br = (int)(bricks[q] % 16);
    for (int l = 0; l < 32; ++l) {
      w->self[l] = t->leaf_of_cell[local_morton_to_cell(b, 32 * br + l)];
      target_position(t, w->self[l], w->tu[l], w->tf[l]);
    }
    walk_brick(w, 0);
    for (int l = 0; l < 32; ++l) {
      phi[32 * q + l] = scale * nm_value(&w->sum[l]);
      if (n_int) n_int[32 * q + l] = w->n_int[l];
      if (n_test) n_test[32 * q + l] = w->n_test[l];
    }
    free(w);
  }
  return OR_OK;
}

/* ------------------------------------------------ learned correction -- */
#define MLP_IN 10
#define MLP_H 64
/* Weights layout (doubles): W1[10][64], b1[64], W2[64][64], b2[64], W3[64], b3. */
#define MLP_NW (MLP_IN * MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1)

static double gelu(double x) {
  const double c = 0.7978845608028654; /* sqrt(2/pi) */
  return 0.5 * x * (1.0 + tanh(c * (x + 0.044715 * x * x * x)));
}

static double mlp_forward(const double *w, const double x[MLP_IN]) {
  const double *W1 = w, *b1 = W1 + MLP_IN * MLP_H, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
  const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
  double h1[MLP_H], h2[MLP_H];
  for (int j = 0; j < MLP_H; ++j) {
    double a = b1[j];
    for (int k = 0; k < MLP_IN; ++k) a += x[k] * W1[k * MLP_H + j];
    h1[j] = gelu(a);
  }
  for (int j = 0; j < MLP_H; ++j) {
    double a = b2[j];
    for (int k = 0; k < MLP_H; ++k) a += h1[k] * W2[k * MLP_H + j];
    h2[j] = gelu(a);
  }
  double y = b3[0];
  for (int k = 0; k < MLP_H; ++k) y += h2[k] * W3[k];
  return y;
}

/* Features of an accepted (target, node) pair: the direction u = d/|d|, the
 * size ratio s = l/|d| and its square and cube, delta/l, the quadrupole
 * along u and its norm, both over M l^2, and s^2 times the former (the
 * leading term of the monopole's error).  Needs the quadrupoles. */
static void pair_features(const onode *n, const double tu[3], double x[MLP_IN], double *s_out,
                          double *mono) {
  double d[3] = {tu[0] - n->R[0], tu[1] - n->R[1], tu[2] - n->R[2]};
  double D = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
  double u[3] = {d[0] / D, d[1] / D, d[2] / D};
  double l = ldexp(1.0, -n->level);
  double s = l / D;
  double ml2 = n->M > 0.0 ? n->M * l * l : 1.0;
  const double *Q = n->Q;
  double quu = Q[0] * u[0] * u[0] + Q[1] * u[1] * u[1] + Q[2] * u[2] * u[2] +
               2.0 * (Q[3] * u[0] * u[1] + Q[4] * u[0] * u[2] + Q[5] * u[1] * u[2]);
  double qf = sqrt(Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2] +
                   2.0 * (Q[3] * Q[3] + Q[4] * Q[4] + Q[5] * Q[5]));
  x[0] = u[0];
  x[1] = u[1];
  x[2] = u[2];
  x[3] = s;
  x[4] = s * s;
  x[5] = s * s * s;
  x[6] = n->delta / l;
  x[7] = quu / ml2;
  x[8] = qf / ml2;
  x[9] = s * s * quu / ml2;
  *s_out = s;
  *mono = n->M / D;
}

typedef struct {
  const otree *t;
  int64_t self;
  float tf[3];
  double tu[3];
  float inv_theta;
  float inv_smin;           /* gate: 1/s_min in binary32, +inf for no gate */
  const double *w;          /* MLP weights (walk) or NULL (pair listing) */
  neumaier sum;
  int64_t n_int, n_test;
  int64_t np, cap;          /* pair listing */
  double *feat, *eps;
  int64_t *node_out;
} learn_state;

/* The gate of the learned correction (not in the paper): an accepted node's
 * term gets the network only while s = l/d >= s_min, decided in binary32 on
 * the opening test's d^2 with the same kind of fixed rounding: corrected iff
 * d2 <= fl(g * g), g = fl(l * fl(1/s_min)).  s_min = 0 (inv_smin = +inf)
 * corrects every accepted node. */
static int gate_f32(const onode *n, const float t[3], float inv_smin) {
  float l = (float)ldexp(1.0, -n->level);
  float g = l * inv_smin;
  float g2 = g * g;
  float dx = t[0] - (float)n->R[0];
  float dy = t[1] - (float)n->R[1];
  float dz = t[2] - (float)n->R[2];
  float d2 = fmaf(dx, dx, fmaf(dz, dz, dy * dy));
  return d2 <= g2;
}

static void walk_learned(learn_state *w, int64_t id) {
  const onode *n = &w->t->node[id];
  if (n->child[0] < 0) {
    if (id != w->self) {
      if (w->w) nm_add(&w->sum, n->M / dist64(w->tu, n->R));
      w->n_int++;
    }
    return;
  }
  w->n_test++;
  if (accept_f32(n, w->tf, w->inv_theta)) {
    double x[MLP_IN], s, mono;
    pair_features(n, w->tu, x, &s, &mono);
    w->n_int++;
    if (w->w) {
      const double corr = gate_f32(n, w->tf, w->inv_smin) ? s * s * mlp_forward(w->w, x) : 0.0;
      nm_add(&w->sum, mono * (1.0 + corr));
    } else {
      if (w->np < w->cap) {
        /* exact contribution of the node: its cells form the pre-order range
           that starts right after it and ends before the next node of the
           same or a shallower level */
        neumaier ex = {0.0, 0.0};
        for (int64_t k = id + 1; k < w->t->nnodes && w->t->node[k].level > n->level; ++k)
          if (w->t->node[k].child[0] < 0)
            nm_add(&ex, w->t->node[k].M / dist64(w->tu, w->t->node[k].R));
        for (int a = 0; a < MLP_IN; ++a) w->feat[MLP_IN * w->np + a] = x[a];
        w->eps[w->np] = nm_value(&ex) / mono - 1.0;
        if (w->node_out) w->node_out[w->np] = id;
      }
      w->np++;
    }
    return;
  }
  for (int o = 0; o < 8; ++o) walk_learned(w, n->child[o]);
}

/* Training pairs of one target: features and eps of every accepted internal
 * node of its per-cell walk.  Returns the number of pairs (the arrays hold
 * the first `cap`), -1 on bad arguments. */
int64_t or_learn_pairs(const void *p, double theta, int64_t target, int64_t cap, double *feat,
                       double *eps, int64_t *node) {
  const otree *t = (const otree *)p;
  if (!check_theta(theta) || !t->have_quad || target < 0 || target >= (int64_t)t->nblocks * 512)
    return -1;
  learn_state w;
  memset(&w, 0, sizeof(w));
  w.t = t;
  w.self = t->leaf_of_cell[target];
  w.inv_theta = (float)(1.0 / theta);
  target_position(t, w.self, w.tu, w.tf);
  w.cap = cap;
  w.feat = feat;
  w.eps = eps;
  w.node_out = node;
  walk_learned(&w, 0);
  return w.np;
}

/* Per-cell walk with the learned correction of every accepted node (of
 * those with s >= s_min when s_min > 0, see gate_f32). */
int or_walk_learned(const void *p, double theta, double G, const double *weights, double s_min,
                    int64_t ntargets, const int64_t *targets, double *phi, int nthreads) {
  const otree *t = (const otree *)p;
  if (!check_theta(theta) || !isfinite(G) || !t->have_quad || !weights || !(s_min >= 0.0) ||
      !(s_min < 1.0))
    return OR_ERR_ARG;
  for (int64_t q = 0; q < ntargets; ++q)
    if (targets[q] < 0 || targets[q] >= (int64_t)t->nblocks * 512) return OR_ERR_ARG;
  float inv_theta = (float)(1.0 / theta);
  double scale = -G / t->L;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
  for (int64_t q = 0; q < ntargets; ++q) {
    learn_state w;
    memset(&w, 0, sizeof(w));
    w.t = t;
    w.self = t->leaf_of_cell[targets[q]];
    w.inv_theta = inv_theta;
    w.inv_smin = s_min > 0.0 ? (float)(1.0 / s_min) : INFINITY;
    w.w = weights;
    target_position(t, w.self, w.tu, w.tf);
    walk_learned(&w, 0);
    phi[q] = scale * nm_value(&w.sum);
  }
  return OR_OK;
}

/* ---------------------------------------------------------- direct sum -- */
/* Eq. 2 without the 1/2: Phi_t = -G sum_{j != t} m_j / |r_t - r_j|. */
int or_direct(const void *p, double G, int64_t ntargets, const int64_t *targets, double *phi,
              int nthreads) {
  const otree *t = (const otree *)p;
  if (!isfinite(G)) return OR_ERR_ARG;
  int64_t ncell = (int64_t)t->nblocks * 512;
  for (int64_t q = 0; q < ntargets; ++q)
    if (targets[q] < 0 || targets[q] >= ncell) return OR_ERR_ARG;
  /* leaves in pre-order */
  int64_t *leaf = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
  if (!leaf) return OR_ERR_OOM;
  int64_t nl = 0;
  for (int64_t id = 0; id < t->nnodes; ++id)
    if (t->node[id].child[0] < 0) leaf[nl++] = id;
  double scale = -G / t->L;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
  for (int64_t q = 0; q < ntargets; ++q) {
    int64_t self = t->leaf_of_cell[targets[q]];
    const double *tu = t->node[self].R;
    neumaier s = {0.0, 0.0};
    for (int64_t j = 0; j < nl; ++j) {
      if (leaf[j] == self) continue;
      const onode *n = &t->node[leaf[j]];
      nm_add(&s, n->M / dist64(tu, n->R));
    }
    phi[q] = scale * nm_value(&s);
  }
  free(leaf);
  return OR_OK;
}

/* Direct sum over an arbitrary set of point masses (positions in any unit):
 * Phi_i = -G sum_{j != i} m_j / |r_i - r_j| for the requested targets. */
int or_direct_points(int64_t n, const double *pos, const double *m, double G,
                     int64_t ntargets, const int64_t *targets, double *phi) {
  for (int64_t q = 0; q < ntargets; ++q) {
    int64_t i = targets[q];
    if (i < 0 || i >= n) return OR_ERR_ARG;
    neumaier s = {0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      nm_add(&s, m[j] / dist64(pos + 3 * i, pos + 3 * j));
    }
    phi[q] = -G * nm_value(&s);
  }
  return OR_OK;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------ periodic boundaries -- */
/*
 * App. A: with periodic boundaries the contribution of a node (or a cell) of
 * mass M to the potential of a cell becomes -G M f(r), f the Ewald field: the
 * potential of a unit mass together with all its periodic copies.  In box
 * units (period 1), splitting 1/r = erf(a r)/r + erfc(a r)/r and summing the
 * smooth erf part over the copies in Fourier space (Eq. ewald), the field of
 * a unit mass at the origin with the box's mean density subtracted (the
 * periodic sum exists only for the density minus its mean) is
 *   psi(r) =  sum_n erfc(a |r + n|) / |r + n|
 *           + (1/pi) sum_{k != 0} exp(-pi^2 |k|^2 / a^2) / |k|^2 cos(2 pi k.r)
 *           - pi / a^2
 * with n and k integer triples whose components lie in [-N, N] (N is the
 * paper's gpuEwaldSeriesN, App. B); the result does not depend on the split
 * parameter a once N is large enough.  The walk uses psi(r) = 1/|r| + chi(r),
 * chi smooth in the box around the origin; in chi the n = 0 real-space term
 * is -erf(a |r|)/|r| (-2 a / sqrt(pi) at r = 0).
 *
 * Table.  The paper keeps the field on grids and interpolates it
 * quadratically in the walk (App. A).  Here chi is tabulated on one grid over
 * the octant [0, 1/2 + h]^3 (chi is even in every coordinate): points
 * (i, j, k) h, h = 1/(2 ng), i, j, k = 0 .. ng + 1, stored at
 * T[(k (ng + 2) + j) (ng + 2) + i].  At u = |displacement| (per component,
 * minimum image, so u <= 1/2) each axis takes the grid index c nearest to
 * u/h, clamped to [1, ng], f = u/h - c, and the three-point Lagrange weights
 * f(f-1)/2, 1 - f^2, f(f+1)/2 of the points c-1, c, c+1; chi(u) is the sum
 * of the 27 products of one weight per axis and the table value.
 *
 * Readings (the paper does not say): the mean density is subtracted; the
 * opening test and the terms use the minimum-image displacement (each
 * component wrapped into [-1/2, 1/2]); a cell also feels the periodic copies
 * of its own mass, m chi(0); in the binary32 test the wrap is
 *   dx = fl(t.x - fl(R.x));  dx > 0.5 -> fl(dx - 1),  dx < -0.5 -> fl(dx + 1)
 * (both exact), then d2 as in the isolated test.
 */
#define EWALD_ALPHA 2.0

/* psi(r) (chi_only = 0) or chi(r) = psi(r) - 1/|r| (chi_only = 1), FP64. */
static double ewald_sum(const double r[3], double a, int N, int chi_only) {
  const double pi = 3.14159265358979323846;
  double real = 0.0, recip = 0.0;
  for (int i = -N; i <= N; ++i)
    for (int j = -N; j <= N; ++j)
      for (int k = -N; k <= N; ++k) {
        double x = r[0] + i, y = r[1] + j, z = r[2] + k;
        double s = sqrt(x * x + y * y + z * z);
        if (i == 0 && j == 0 && k == 0 && chi_only)
          real += s > 0.0 ? -erf(a * s) / s : -2.0 * a / sqrt(pi);
        else
          real += erfc(a * s) / s;
      }
  for (int i = -N; i <= N; ++i)
    for (int j = -N; j <= N; ++j)
      for (int k = -N; k <= N; ++k) {
        if (i == 0 && j == 0 && k == 0) continue;
        double k2 = (double)(i * i + j * j + k * k);
        double kr = i * r[0] + j * r[1] + k * r[2];
        recip += exp(-pi * pi * k2 / (a * a)) / k2 * cos(2.0 * pi * kr);
      }
  return real + recip / pi - pi / (a * a);
}

/* psi or chi at n points r[3n] (box units), split parameter a, range N. */
int or_ewald_sum(int64_t n, const double *r, double a, int N, int chi_only, double *out) {
  if (n < 0 || !(a > 0.0) || N < 0) return OR_ERR_ARG;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t q = 0; q < n; ++q) out[q] = ewald_sum(r + 3 * q, a, N, chi_only);
  return OR_OK;
}

/* The table of chi (see above): (ng + 2)^3 values, a = EWALD_ALPHA. */
int or_ewald_table(int ng, int N, double *T) {
  if (ng < 2 || N < 1) return OR_ERR_ARG;
  const int m = ng + 2;
  const double h = 1.0 / (2.0 * ng);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64)
#endif
  for (int64_t q = 0; q < (int64_t)m * m * m; ++q) {
    int i = (int)(q % m), j = (int)((q / m) % m), k = (int)(q / ((int64_t)m * m));
    double r[3] = {i * h, j * h, k * h};
    T[q] = ewald_sum(r, EWALD_ALPHA, N, 1);
  }
  return OR_OK;
}

/* Quadratic interpolation of the table at u (u >= 0 per component). */
static double ewald_interp(const double *T, int ng, const double u[3]) {
  const int m = ng + 2;
  int c[3];
  double w[3][3];
  for (int a = 0; a < 3; ++a) {
    double t = u[a] * (2.0 * ng);
    int ci = (int)floor(t + 0.5);
    if (ci < 1) ci = 1;
    if (ci > ng) ci = ng;
    double f = t - ci;
    w[a][0] = 0.5 * f * (f - 1.0);
    w[a][1] = 1.0 - f * f;
    w[a][2] = 0.5 * f * (f + 1.0);
    c[a] = ci;
  }
  double s = 0.0;
  for (int kz = 0; kz < 3; ++kz)
    for (int jy = 0; jy < 3; ++jy)
      for (int ix = 0; ix < 3; ++ix)
        s += w[2][kz] * w[1][jy] * w[0][ix] *
             T[((int64_t)(c[2] - 1 + kz) * m + (c[1] - 1 + jy)) * m + (c[0] - 1 + ix)];
  return s;
}

int or_ewald_interp(const double *T, int ng, int64_t n, const double *u, double *out) {
  if (ng < 2 || n < 0) return OR_ERR_ARG;
  for (int64_t q = 0; q < n; ++q) {
    double v[3] = {fabs(u[3 * q]), fabs(u[3 * q + 1]), fabs(u[3 * q + 2])};
    if (v[0] > 0.5 + 0.5 / ng || v[1] > 0.5 + 0.5 / ng || v[2] > 0.5 + 0.5 / ng)
      return OR_ERR_ARG;
    out[q] = ewald_interp(T, ng, v);
  }
  return OR_OK;
}

static double wrap64(double d) {
  if (d > 0.5) return d - 1.0;
  if (d < -0.5) return d + 1.0;
  return d;
}
static float wrap32(float d) {
  if (d > 0.5f) return d - 1.0f;
  if (d < -0.5f) return d + 1.0f;
  return d;
}

/* The binary32 test of Eq. 4 on the minimum-image displacement. */
static int accept_f32_periodic(const onode *n, const float t[3], float inv_theta) {
  float l = (float)ldexp(1.0, -n->level);
  float s = l * inv_theta;
  s = s + (float)n->delta;
  float s2 = s * s;
  float dx = wrap32(t[0] - (float)n->R[0]);
  float dy = wrap32(t[1] - (float)n->R[1]);
  float dz = wrap32(t[2] - (float)n->R[2]);
  float d2 = fmaf(dx, dx, fmaf(dz, dz, dy * dy));
  return d2 > s2;
}

/* M psi(r_t - R) with psi = 1/d + chi from the table (T) or from the sum
 * (T == NULL, range N), minimum image; for the target's own cell (self) the
 * copies only: M chi(0). */
static double periodic_term(double M, const double tu[3], const double R[3], int self,
                            const double *T, int ng, int N) {
  double x[3] = {wrap64(tu[0] - R[0]), wrap64(tu[1] - R[1]), wrap64(tu[2] - R[2])};
  if (self) x[0] = x[1] = x[2] = 0.0;
  double chi;
  if (T) {
    double u[3] = {fabs(x[0]), fabs(x[1]), fabs(x[2])};
    chi = ewald_interp(T, ng, u);
  } else {
    chi = ewald_sum(x, EWALD_ALPHA, N, 1);
  }
  if (self) return M * chi;
  double d = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
  return M * (1.0 / d + chi);
}

typedef struct {
  const otree *t;
  int64_t self;
  float tf[3];
  double tu[3];
  float inv_theta;
  const double *T;
  int ng;
  neumaier sum;
  int64_t n_int, n_test;
} pwalk_state;

static void walk_periodic(pwalk_state *w, int64_t id) {
  const onode *n = &w->t->node[id];
  if (n->child[0] < 0) {                      /* a leaf cell, or the target's own */
    nm_add(&w->sum, periodic_term(n->M, w->tu, n->R, id == w->self, w->T, w->ng, 0));
    if (id != w->self) w->n_int++;
    return;
  }
  w->n_test++;
  if (accept_f32_periodic(n, w->tf, w->inv_theta)) {
    nm_add(&w->sum, periodic_term(n->M, w->tu, n->R, 0, w->T, w->ng, 0));
    w->n_int++;
    return;
  }
  for (int o = 0; o < 8; ++o) walk_periodic(w, n->child[o]);
}

/* Per-cell walk with periodic boundaries (App. A): minimum-image test and
 * terms M (1/d + chi(d)) with chi interpolated from the table T (ng). */
int or_walk_periodic(const void *p, double theta, double G, const double *T, int ng,
                     int64_t ntargets, const int64_t *targets, double *phi, int64_t *n_int,
                     int64_t *n_test, int nthreads) {
  const otree *t = (const otree *)p;
  if (!check_theta(theta) || !isfinite(G) || !T || ng < 2) return OR_ERR_ARG;
  int64_t ncell = (int64_t)t->nblocks * 512;
  for (int64_t q = 0; q < ntargets; ++q)
    if (targets[q] < 0 || targets[q] >= ncell) return OR_ERR_ARG;
  float inv_theta = (float)(1.0 / theta);
  double scale = -G / t->L;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
  for (int64_t q = 0; q < ntargets; ++q) {
    pwalk_state w;
    memset(&w, 0, sizeof(w));
    w.t = t;
    w.self = t->leaf_of_cell[targets[q]];
    w.inv_theta = inv_theta;
    w.T = T;
    w.ng = ng;
    target_position(t, w.self, w.tu, w.tf);
    walk_periodic(&w, 0);
    phi[q] = scale * nm_value(&w.sum);
    if (n_int) n_int[q] = w.n_int;
    if (n_test) n_test[q] = w.n_test;
  }
  return OR_OK;
}

/* Direct periodic sum: Phi_t = -(G/L) (sum_{j != t} m_j psi(r_t - r_j)
 * + m_t chi(0)), psi from the table T (ng) or, with T == NULL, from the
 * Ewald sum itself (range N, split EWALD_ALPHA). */
int or_direct_periodic(const void *p, double G, const double *T, int ng, int N,
                       int64_t ntargets, const int64_t *targets, double *phi, int nthreads) {
  const otree *t = (const otree *)p;
  if (!isfinite(G) || (T && ng < 2) || (!T && N < 1)) return OR_ERR_ARG;
  int64_t ncell = (int64_t)t->nblocks * 512;
  for (int64_t q = 0; q < ntargets; ++q)
    if (targets[q] < 0 || targets[q] >= ncell) return OR_ERR_ARG;
  int64_t *leaf = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
  if (!leaf) return OR_ERR_OOM;
  int64_t nl = 0;
  for (int64_t id = 0; id < t->nnodes; ++id)
    if (t->node[id].child[0] < 0) leaf[nl++] = id;
  double scale = -G / t->L;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t q = 0; q < ntargets; ++q) {
    int64_t self = t->leaf_of_cell[targets[q]];
    const double *tu = t->node[self].R;
    neumaier s = {0.0, 0.0};
    for (int64_t j = 0; j < nl; ++j) {
      const onode *n = &t->node[leaf[j]];
      nm_add(&s, periodic_term(n->M, tu, n->R, leaf[j] == self, T, ng, N));
    }
    phi[q] = scale * nm_value(&s);
  }
  free(leaf);
  return OR_OK;
}
