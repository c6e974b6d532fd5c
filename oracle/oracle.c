/*
 * oracle.c -- plain, serial, FP64 CPU reference for the discrete Eikonal
 * system solved by the parallel Heap-Cell Method (Chacon & Vladimirsky,
 * "A parallel Heap-Cell Method for Eikonal equations", arXiv:1306.4743).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load it.  It shares no code, header or constant with the CUDA library.
 *
 * What is computed (Sec. 1.1, Eq. 2): on a uniform grid x_ijk = (ih,jh,kh),
 * 0 <= i < nx, 0 <= j < ny, 0 <= k < nz, the vector U with
 *   U = q on the exit nodes Q' (fixed, never recomputed), and at every
 *   other node
 *   sum over axes d of ( max(D^-d U, -D^+d U, 0) )^2 = 1 / F^2,
 * where every value outside the grid is +infinity (Sec. 1.1).
 * Multiplying by h^2 and writing a_d = min(U at the two axis-d neighbours),
 * s = h / F, the equation at one node reads
 *   sum_d ( max(U - a_d, 0) )^2 = s^2                       (*)
 * which has exactly one root U > min_d a_d when some a_d is finite; that
 * root is the local solve Lambda(U) used by every method in the paper
 * (Alg. 2, "solve equation (2)").  The grid solution is the fixed point of
 * U_x <- min(U_x, Lambda_x(U)) started from +infinity off Q'.
 *
 * Index convention: node (i,j,k) lives at i + nx*(j + ny*k) (i fastest).
 * F is float (the library's input type); every step here is in double:
 * s = h / (double)F.
 *
 * Functions:
 *   orc_local_solve           root of (*) by sorting a and trying 1, 2, 3 terms
 *   orc_local_solve_textbook  the same root from the unshifted quadratic
 *   orc_fmm                   Fast Marching Method with a binary heap (Sec. 2)
 *   orc_value_iteration       Jacobi iteration of the fixed-point map from +inf
 *   orc_gauss_seidel_perm     Gauss-Seidel passes in a caller-given node order
 *   orc_fsm                   Fast Sweeping (Sec. 2): 8 lexicographic loop
 *                             orderings, with per-sweep statistics (Tables 4-6)
 *   orc_residual              max |U - Lambda(U)| over non-exit nodes
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 3

static inline int64_t node_index(int64_t i, int64_t j, int64_t k, int64_t nx,
                                 int64_t ny) {
  return i + nx * (j + ny * k);
}

/* ------------------------------------------------------------------------ */
/* Local solve of (*).  Sort a1 <= a2 <= a3; the root uses the m smallest
 * values for the first m in {1,2,3} whose root does not exceed a_{m+1}.
 * Writing U = a1 + w and b_d = a_d - a1 (the same equation, shifted so that
 * every term is of the size of s):
 *   m = 1:  w = s
 *   m = 2:  w^2 + (w - b)^2 = s^2           ->  w = (b + sqrt(2 s^2 - b^2)) / 2
 *   m = 3:  w^2 + (w-b2)^2 + (w-b3)^2 = s^2 ->  w = (p + sqrt(p^2 - 3(b2^2 + b3^2 - s^2))) / 3,
 *           p = b2 + b3
 * (the larger root in each case: U must exceed every a_d it uses). */
double orc_local_solve(double ax, double ay, double az, double s) {
  double a1 = ax, a2 = ay, a3 = az, t;
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (a2 > a3) { t = a2; a2 = a3; a3 = t; }
  if (a1 > a2) { t = a1; a1 = a2; a2 = t; }
  if (isinf(a1)) return INFINITY; /* no finite neighbour: no information */
  double u = a1 + s;
  if (u <= a2) return u;
  double b = a2 - a1;
  double disc2 = 2.0 * s * s - b * b;
  if (disc2 < 0.0) disc2 = 0.0; /* cannot happen in exact arithmetic (b < s) */
  u = a1 + 0.5 * (b + sqrt(disc2));
  if (u <= a3) return u;
  double b2 = a2 - a1, b3 = a3 - a1, p = b2 + b3;
  double disc3 = p * p - 3.0 * (b2 * b2 + b3 * b3 - s * s);
  if (disc3 < 0.0) disc3 = 0.0; /* cannot happen in exact arithmetic */
  return a1 + (p + sqrt(disc3)) / 3.0;
}

/* The same root written from the unshifted quadratic
 *   m U^2 - 2 (sum a) U + (sum a^2 - s^2) = 0
 * over the m smallest a.  Used only to cross-check orc_local_solve; it loses
 * digits to cancellation when a >> s. */
double orc_local_solve_textbook(double ax, double ay, double az, double s) {
  double a[3] = {ax, ay, az}, t;
  if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
  if (a[1] > a[2]) { t = a[1]; a[1] = a[2]; a[2] = t; }
  if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
  if (isinf(a[0])) return INFINITY;
  double u = INFINITY;
  for (int m = 1; m <= 3; ++m) {
    if (isinf(a[m - 1])) break;
    double sa = 0.0, sa2 = 0.0;
    for (int d = 0; d < m; ++d) { sa += a[d]; sa2 += a[d] * a[d]; }
    double disc = sa * sa - m * (sa2 - s * s);
    if (disc < 0.0) disc = 0.0;
    u = (sa + sqrt(disc)) / m;
    if (m == 3 || u <= a[m]) break;
  }
  return u;
}

/* a_d for node (i,j,k) from the array V; off-grid neighbours are +inf. */
static inline void axis_minima(const double *V, int64_t i, int64_t j,
                               int64_t k, int64_t nx, int64_t ny, int64_t nz,
                               double *ax, double *ay, double *az) {
  int64_t c = node_index(i, j, k, nx, ny);
  double m = INFINITY;
  if (i > 0 && V[c - 1] < m) m = V[c - 1];
  if (i + 1 < nx && V[c + 1] < m) m = V[c + 1];
  *ax = m;
  m = INFINITY;
  if (j > 0 && V[c - nx] < m) m = V[c - nx];
  if (j + 1 < ny && V[c + nx] < m) m = V[c + nx];
  *ay = m;
  m = INFINITY;
  if (k > 0 && V[c - nx * ny] < m) m = V[c - nx * ny];
  if (k + 1 < nz && V[c + nx * ny] < m) m = V[c + nx * ny];
  *az = m;
}

static int check_inputs(int64_t nx, int64_t ny, int64_t nz, double h,
                        const float *F, const uint8_t *mask, const double *q) {
  if (nx < 1 || ny < 1 || nz < 1 || !(h > 0.0) || isinf(h)) return ORC_EINVAL;
  int64_t M = nx * ny * nz, nsrc = 0;
  for (int64_t x = 0; x < M; ++x) {
    if (mask[x]) {
      if (!isfinite(q[x])) return ORC_EINVAL;
      ++nsrc;
    } else if (!(F[x] > 0.0f) || isinf(F[x])) {
      return ORC_EINVAL;
    }
  }
  return nsrc > 0 ? ORC_OK : ORC_EINVAL;
}

/* ------------------------------------------------------------------------ */
/* Fast Marching Method (Sec. 2): the "considered" node with the smallest
 * temporary value is accepted; each not-yet-accepted neighbour y is then
 * recomputed from accepted values only (others count as +inf) and keeps
 * the smaller of its old and new values.  Exit nodes enter the heap with
 * their value q and are never recomputed, so exit values need not be equal.
 * Binary min-heap with a position table for decrease-key. */
typedef struct {
  int64_t *heap; /* node ids */
  int64_t *pos;  /* heap slot of each node, -1 if not in heap */
  int64_t size;
  const double *key;
} orc_heap;

static void heap_swap(orc_heap *H, int64_t a, int64_t b) {
  int64_t na = H->heap[a], nb = H->heap[b];
  H->heap[a] = nb; H->heap[b] = na;
  H->pos[nb] = a; H->pos[na] = b;
}
static void heap_up(orc_heap *H, int64_t p) {
  while (p > 0) {
    int64_t parent = (p - 1) / 2;
    if (H->key[H->heap[parent]] <= H->key[H->heap[p]]) break;
    heap_swap(H, p, parent);
    p = parent;
  }
}
static void heap_down(orc_heap *H, int64_t p) {
  for (;;) {
    int64_t l = 2 * p + 1, r = l + 1, m = p;
    if (l < H->size && H->key[H->heap[l]] < H->key[H->heap[m]]) m = l;
    if (r < H->size && H->key[H->heap[r]] < H->key[H->heap[m]]) m = r;
    if (m == p) break;
    heap_swap(H, p, m);
    p = m;
  }
}
static void heap_push(orc_heap *H, int64_t node) {
  H->heap[H->size] = node;
  H->pos[node] = H->size;
  H->size++;
  heap_up(H, H->size - 1);
}
static int64_t heap_pop(orc_heap *H) {
  int64_t top = H->heap[0];
  H->size--;
  if (H->size > 0) {
    H->heap[0] = H->heap[H->size];
    H->pos[H->heap[0]] = 0;
    heap_down(H, 0);
  }
  H->pos[top] = -1;
  return top;
}

int orc_fmm(int64_t nx, int64_t ny, int64_t nz, double h, const float *F,
            const uint8_t *mask, const double *q, double *U,
            int64_t *n_recompute) {
  int rc = check_inputs(nx, ny, nz, h, F, mask, q);
  if (rc) return rc;
  int64_t M = nx * ny * nz;
  uint8_t *accepted = (uint8_t *)calloc((size_t)M, 1);
  double *Acc = (double *)malloc((size_t)M * sizeof(double)); /* accepted values, +inf otherwise */
  orc_heap H;
  H.heap = (int64_t *)malloc((size_t)M * sizeof(int64_t));
  H.pos = (int64_t *)malloc((size_t)M * sizeof(int64_t));
  H.size = 0;
  H.key = U;
  if (!accepted || !Acc || !H.heap || !H.pos) {
    free(accepted); free(Acc); free(H.heap); free(H.pos);
    return ORC_ENOMEM;
  }
  for (int64_t x = 0; x < M; ++x) {
    U[x] = INFINITY;
    Acc[x] = INFINITY;
    H.pos[x] = -1;
  }
  for (int64_t x = 0; x < M; ++x)
    if (mask[x]) { U[x] = q[x]; heap_push(&H, x); }
  int64_t recompute = 0;
  while (H.size > 0) {
    int64_t x = heap_pop(&H);
    accepted[x] = 1;
    Acc[x] = U[x];
    int64_t k = x / (nx * ny), j = (x / nx) % ny, i = x % nx;
    int64_t nb[6];
    int nn = 0;
    if (i > 0) nb[nn++] = x - 1;
    if (i + 1 < nx) nb[nn++] = x + 1;
    if (j > 0) nb[nn++] = x - nx;
    if (j + 1 < ny) nb[nn++] = x + nx;
    if (k > 0) nb[nn++] = x - nx * ny;
    if (k + 1 < nz) nb[nn++] = x + nx * ny;
    for (int t = 0; t < nn; ++t) {
      int64_t y = nb[t];
      if (accepted[y] || mask[y]) continue;
      int64_t yk = y / (nx * ny), yj = (y / nx) % ny, yi = y % nx;
      double ax, ay, az;
      axis_minima(Acc, yi, yj, yk, nx, ny, nz, &ax, &ay, &az);
      double v = orc_local_solve(ax, ay, az, h / (double)F[y]);
      ++recompute;
      if (v < U[y]) {
        U[y] = v;
        if (H.pos[y] >= 0) heap_up(&H, H.pos[y]);
        else heap_push(&H, y);
      }
    }
  }
  if (n_recompute) *n_recompute = recompute;
  free(accepted); free(Acc); free(H.heap); free(H.pos);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Jacobi value iteration: V^{m+1}_x = min(V^m_x, Lambda_x(V^m)) at every
 * non-exit node, all from the previous iterate, from V^0 = +inf off Q',
 * until an iteration changes no bit.  Brute force for tiny grids. */
int orc_value_iteration(int64_t nx, int64_t ny, int64_t nz, double h,
                        const float *F, const uint8_t *mask, const double *q,
                        double *U, int64_t max_iter, int64_t *iters) {
  int rc = check_inputs(nx, ny, nz, h, F, mask, q);
  if (rc) return rc;
  int64_t M = nx * ny * nz;
  double *V = (double *)malloc((size_t)M * sizeof(double));
  if (!V) return ORC_ENOMEM;
  for (int64_t x = 0; x < M; ++x) U[x] = mask[x] ? q[x] : INFINITY;
  int64_t it = 0;
  int changed = 1;
  while (changed && it < max_iter) {
    changed = 0;
    memcpy(V, U, (size_t)M * sizeof(double));
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
          int64_t x = node_index(i, j, k, nx, ny);
          if (mask[x]) continue;
          double ax, ay, az;
          axis_minima(V, i, j, k, nx, ny, nz, &ax, &ay, &az);
          double v = orc_local_solve(ax, ay, az, h / (double)F[x]);
          if (v < V[x]) { U[x] = v; changed = 1; }
        }
    ++it;
  }
  free(V);
  if (iters) *iters = it;
  return changed ? ORC_ENOCONV : ORC_OK;
}

/* Gauss-Seidel: passes over the nodes in the order perm[0..M-1], updating
 * in place with U_x <- min(U_x, Lambda_x(U)), until a pass changes no bit. */
int orc_gauss_seidel_perm(int64_t nx, int64_t ny, int64_t nz, double h,
                          const float *F, const uint8_t *mask,
                          const double *q, const int64_t *perm, double *U,
                          int64_t max_pass, int64_t *passes) {
  int rc = check_inputs(nx, ny, nz, h, F, mask, q);
  if (rc) return rc;
  int64_t M = nx * ny * nz;
  for (int64_t x = 0; x < M; ++x) U[x] = mask[x] ? q[x] : INFINITY;
  int64_t it = 0;
  int changed = 1;
  while (changed && it < max_pass) {
    changed = 0;
    for (int64_t t = 0; t < M; ++t) {
      int64_t x = perm[t];
      if (mask[x]) continue;
      int64_t k = x / (nx * ny), j = (x / nx) % ny, i = x % nx;
      double ax, ay, az;
      axis_minima(U, i, j, k, nx, ny, nz, &ax, &ay, &az);
      double v = orc_local_solve(ax, ay, az, h / (double)F[x]);
      if (v < U[x]) { U[x] = v; changed = 1; }
    }
    ++it;
  }
  if (passes) *passes = it;
  return changed ? ORC_ENOCONV : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Fast Sweeping (Sec. 2): Gauss-Seidel over the whole grid in the 2^3
 * lexicographic loop orderings, taken from dir_order[] cyclically.  A
 * direction code d in 0..7 sweeps i upward when bit 0 is clear (downward
 * when set), j by bit 1, k by bit 2.  `inner` names the fastest-running
 * loop axis (0 = i, 2 = k; the other two nest as (k, j, i) minus inner).
 * `unreached` is the stand-in for +inf in the stored values (the paper's
 * tables show a finite 1e9 sentinel, Tables 4-5; pass INFINITY for the
 * mathematical definition).  A node counts as changed in a sweep when its
 * value decreases by more than kappa; sweeping stops after the first sweep
 * with no such node.  Per-sweep maximum decrease and changed-node count are
 * written to max_change[s] and n_changed[s] for s < max_sweeps. */
int orc_fsm(int64_t nx, int64_t ny, int64_t nz, double h, const float *F,
            const uint8_t *mask, const double *q, const int *dir_order,
            int n_dir, int inner, double unreached, double kappa,
            int64_t max_sweeps, double *U, int64_t *sweeps,
            double *max_change, int64_t *n_changed) {
  int rc = check_inputs(nx, ny, nz, h, F, mask, q);
  if (rc) return rc;
  if (n_dir < 1 || inner < 0 || inner > 2) return ORC_EINVAL;
  int64_t M = nx * ny * nz;
  int64_t n[3] = {nx, ny, nz};
  for (int64_t x = 0; x < M; ++x) U[x] = mask[x] ? q[x] : unreached;
  /* loop axes from outermost to innermost */
  int order[3];
  {
    int t = 0;
    for (int a = 2; a >= 0; --a)
      if (a != inner) order[t++] = a;
    order[2] = inner;
  }
  int64_t s = 0;
  for (;;) {
    if (s >= max_sweeps) { if (sweeps) *sweeps = s; return ORC_ENOCONV; }
    int d = dir_order[s % n_dir];
    double mc = 0.0;
    int64_t nc = 0;
    int64_t c[3];
    int64_t lo[3], st[3];
    for (int a = 0; a < 3; ++a) {
      int down = (d >> a) & 1;
      lo[a] = down ? n[a] - 1 : 0;
      st[a] = down ? -1 : 1;
    }
    for (int64_t t0 = 0; t0 < n[order[0]]; ++t0) {
      c[order[0]] = lo[order[0]] + st[order[0]] * t0;
      for (int64_t t1 = 0; t1 < n[order[1]]; ++t1) {
        c[order[1]] = lo[order[1]] + st[order[1]] * t1;
        for (int64_t t2 = 0; t2 < n[order[2]]; ++t2) {
          c[order[2]] = lo[order[2]] + st[order[2]] * t2;
          int64_t x = node_index(c[0], c[1], c[2], nx, ny);
          if (mask[x]) continue;
          double ax, ay, az;
          axis_minima(U, c[0], c[1], c[2], nx, ny, nz, &ax, &ay, &az);
          double v = orc_local_solve(ax, ay, az, h / (double)F[x]);
          if (v < U[x]) {
            double dv = U[x] - v;
            U[x] = v;
            if (dv > kappa) {
              ++nc;
              if (dv > mc) mc = dv;
            }
          }
        }
      }
    }
    if (max_change) max_change[s] = mc;
    if (n_changed) n_changed[s] = nc;
    ++s;
    if (nc == 0) break;
  }
  if (sweeps) *sweeps = s;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Residual of the fixed point: max over non-exit nodes of |U - Lambda(U)|
 * (Lambda from all six neighbours of U).  Also counts non-finite values. */
double orc_residual(int64_t nx, int64_t ny, int64_t nz, double h,
                    const float *F, const uint8_t *mask, const double *U,
                    int64_t *n_nonfinite) {
  double r = 0.0;
  int64_t bad = 0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t x = node_index(i, j, k, nx, ny);
        if (!isfinite(U[x])) { ++bad; continue; }
        if (mask[x]) continue;
        double ax, ay, az;
        axis_minima(U, i, j, k, nx, ny, nz, &ax, &ay, &az);
        double v = orc_local_solve(ax, ay, az, h / (double)F[x]);
        double e = fabs(U[x] - v);
        if (e > r) r = e;
      }
  if (n_nonfinite) *n_nonfinite = bad;
  return r;
}
