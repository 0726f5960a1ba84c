/*
 * ctiled.c -- the paper's own design on the host: tiled QR with the four
 * tile kernels of Section 3.1 (GEQRT, LARFB, TSQRT, SSRFB, with inner
 * blocking ib), driven by dynamic scheduling of Algorithm 1's task DAG over
 * POSIX threads (Section 3.3).
 *
 * TEST INFRASTRUCTURE ONLY: part of the oracle.  It is the multithreaded CPU
 * baseline of the benchmark and a second, independent implementation that
 * the tests compare with the NumPy oracle (oracle/tiled.py).  Nothing in the
 * product package uses it, and it shares no code with the CUDA path.
 *
 * Plain C99, float64, no BLAS: every kernel is written as the loops of its
 * definition.  Conventions (the readings the NumPy oracle records too):
 *  - reflectors in the LAPACK convention (Section 2 takes them from the
 *    textbooks): beta = -sign(alpha) ||x||, sign(0) = +1,
 *    tau = (beta - alpha) / beta, v = [1; x2 / (alpha - beta)];
 *    ||x2|| = 0 gives tau = 0;
 *  - T by the forward columnwise recurrence T[i,i] = tau_i,
 *    T[0:i,i] = -tau_i T[0:i,0:i] (V[:,0:i]^T v_i), one ib x ib block per
 *    inner block, stored side by side (ib x nb per tile), so the
 *    factorization applies Q^T = I - V T^T V^T;
 *  - block l of a TSQRT touches rows l*ib .. (l+1)*ib-1 of the top triangle
 *    and all rows of the bottom tile;
 *  - A is zero-padded to whole tiles (Block Data Layout, Section 3.4).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef struct {
  int p, q, nb, ib;
  double* tiles; /* tile (i, j) at (i + j p) nb^2, column-major, ld nb */
  double* T;     /* ib x nb per (i, k), k < min(p, q), i >= k */
} grid_t;

static double* tile(const grid_t* g, int i, int j) {
  return g->tiles + ((size_t)i + (size_t)j * g->p) * (size_t)g->nb * g->nb;
}

static double* tblock(const grid_t* g, int i, int k) {
  const size_t off = (size_t)k * g->p - (size_t)k * (k - 1) / 2 + (size_t)(i - k);
  return g->T + off * (size_t)g->ib * g->nb;
}

/* ||x||_2 scaled by max |x_i| so nothing overflows or underflows. */
static double scaled_norm(const double* x, int n) {
  double s = 0.0, t = 0.0;
  for (int r = 0; r < n; ++r) {
    const double a = fabs(x[r]);
    if (a > s) s = a;
  }
  if (s == 0.0 || !isfinite(s)) return s;
  for (int r = 0; r < n; ++r) {
    const double y = x[r] / s;
    t += y * y;
  }
  return s * sqrt(t);
}

/* Reflector H = I - tau [1; v2][1; v2]^T with H [alpha; x2] = [beta; 0]
 * (Section 2, DGEQR2 step): *alpha becomes beta, x2 becomes v2. */
static double reflector(double* alpha, double* x2, int n) {
  const double xn = scaled_norm(x2, n);
  if (xn == 0.0) return 0.0;
  const double a = *alpha;
  const double nrm = hypot(a, xn);
  const double beta = a >= 0.0 ? -nrm : nrm;
  const double tau = (beta - a) / beta;
  const double s = 1.0 / (a - beta);
  for (int r = 0; r < n; ++r) x2[r] *= s;
  *alpha = beta;
  return tau;
}

/* T_l from the taus and the Gram entries z[a] = v_a^T v_i (forward
 * columnwise recurrence).  Tl is ib x ib column-major with leading
 * dimension ib (a block of the ib x nb T array). */
static void form_t_column(double* Tl, int ib, int i, double tau, const double* z) {
  Tl[i + (size_t)i * ib] = tau;
  for (int a = 0; a < i; ++a) {
    double s = 0.0;
    for (int b = a; b < i; ++b) s += Tl[a + (size_t)b * ib] * z[b];
    Tl[a + (size_t)i * ib] = -tau * s;
  }
}

/* w <- T_l^T w for upper triangular T_l (ib x ib, ld ib). */
static void apply_tt(const double* Tl, int ib, double* w) {
  for (int a = ib - 1; a >= 0; --a) {
    double s = 0.0;
    for (int b = 0; b <= a; ++b) s += Tl[b + (size_t)a * ib] * w[b];
    w[a] = s;
  }
}

/* GEQRT (DGEQT2 with inner blocking, Section 3.1): QR of the diagonal tile
 * A (nb x nb); R on and above the diagonal, V below it, T (ib x nb). */
static void geqrt(double* A, double* T, int nb, int ib) {
  double tau[64], z[64], w[64];
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const int l1 = l0 + ib;
    double* Tl = T + (size_t)l0 * ib;
    for (int c = l0; c < l1; ++c) {
      double* vc = A + (size_t)c * nb;
      const double t = reflector(&vc[c], &vc[c + 1], nb - c - 1);
      tau[c - l0] = t;
      if (t != 0.0)
        for (int j = c + 1; j < l1; ++j) {
          double* aj = A + (size_t)j * nb;
          double s = aj[c];
          for (int r = c + 1; r < nb; ++r) s += vc[r] * aj[r];
          aj[c] -= t * s;
          for (int r = c + 1; r < nb; ++r) aj[r] -= t * s * vc[r];
        }
    }
    for (int i = 0; i < ib; ++i) {
      const double* vi = A + (size_t)(l0 + i) * nb;
      for (int a = 0; a < i; ++a) {
        const double* va = A + (size_t)(l0 + a) * nb;
        double s = va[l0 + i];              /* v_i has 1 at row l0 + i */
        for (int r = l0 + i + 1; r < nb; ++r) s += va[r] * vi[r];
        z[a] = s;
      }
      form_t_column(Tl, ib, i, tau[i], z);
    }
    /* trailing columns: c_j <- (I - V T_l^T V^T) c_j */
    for (int j = l1; j < nb; ++j) {
      double* cj = A + (size_t)j * nb;
      for (int a = 0; a < ib; ++a) {
        const double* va = A + (size_t)(l0 + a) * nb;
        double s = cj[l0 + a];
        for (int r = l0 + a + 1; r < nb; ++r) s += va[r] * cj[r];
        w[a] = s;
      }
      apply_tt(Tl, ib, w);
      for (int a = 0; a < ib; ++a) {
        const double* va = A + (size_t)(l0 + a) * nb;
        cj[l0 + a] -= w[a];
        for (int r = l0 + a + 1; r < nb; ++r) cj[r] -= va[r] * w[a];
      }
    }
  }
}

/* LARFB (Section 3.1): C (nb x nb) <- Q_kk^T C with the reflectors of a
 * GEQRT'ed diagonal tile V (unit lower part) and T, blocks l = 0, 1, .... */
static void larfb(const double* V, const double* T, double* C, int nb, int ib) {
  double w[64];
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const double* Tl = T + (size_t)l0 * ib;
    for (int j = 0; j < nb; ++j) {
      double* cj = C + (size_t)j * nb;
      for (int a = 0; a < ib; ++a) {
        const double* va = V + (size_t)(l0 + a) * nb;
        double s = cj[l0 + a];
        for (int r = l0 + a + 1; r < nb; ++r) s += va[r] * cj[r];
        w[a] = s;
      }
      apply_tt(Tl, ib, w);
      for (int a = 0; a < ib; ++a) {
        const double* va = V + (size_t)(l0 + a) * nb;
        cj[l0 + a] -= w[a];
        for (int r = l0 + a + 1; r < nb; ++r) cj[r] -= va[r] * w[a];
      }
    }
  }
}

/* TSQRT (DTSQT2 with inner blocking, Section 3.1): QR of the upper triangle
 * R of the diagonal tile stacked on B (nb x nb); R's upper triangle becomes
 * the new R, B becomes V, T (ib x nb).  The strictly lower part of R (V_kk)
 * is not touched. */
static void tsqrt(double* R, double* B, double* T, int nb, int ib) {
  double tau[64], z[64], w[64];
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const int l1 = l0 + ib;
    double* Tl = T + (size_t)l0 * ib;
    for (int c = l0; c < l1; ++c) {
      double* bc = B + (size_t)c * nb;
      const double t = reflector(&R[c + (size_t)c * nb], bc, nb);
      tau[c - l0] = t;
      if (t != 0.0)
        for (int j = c + 1; j < l1; ++j) {
          double* bj = B + (size_t)j * nb;
          double s = R[c + (size_t)j * nb];
          for (int r = 0; r < nb; ++r) s += bc[r] * bj[r];
          R[c + (size_t)j * nb] -= t * s;
          for (int r = 0; r < nb; ++r) bj[r] -= t * s * bc[r];
        }
    }
    /* the top parts of the block's reflectors are distinct unit vectors, so
     * v_a^T v_i is the product of their bottom parts */
    for (int i = 0; i < ib; ++i) {
      const double* bi = B + (size_t)(l0 + i) * nb;
      for (int a = 0; a < i; ++a) {
        const double* ba = B + (size_t)(l0 + a) * nb;
        double s = 0.0;
        for (int r = 0; r < nb; ++r) s += ba[r] * bi[r];
        z[a] = s;
      }
      form_t_column(Tl, ib, i, tau[i], z);
    }
    for (int j = l1; j < nb; ++j) {
      double* bj = B + (size_t)j * nb;
      for (int a = 0; a < ib; ++a) {
        const double* ba = B + (size_t)(l0 + a) * nb;
        double s = R[l0 + a + (size_t)j * nb];
        for (int r = 0; r < nb; ++r) s += ba[r] * bj[r];
        w[a] = s;
      }
      apply_tt(Tl, ib, w);
      for (int a = 0; a < ib; ++a) {
        const double* ba = B + (size_t)(l0 + a) * nb;
        R[l0 + a + (size_t)j * nb] -= w[a];
        for (int r = 0; r < nb; ++r) bj[r] -= ba[r] * w[a];
      }
    }
  }
}

/* SSRFB (Section 3.1): [Ck; Ci] <- Q^T [Ck; Ci] with the reflectors [I; V]
 * and T of a TSQRT, blocks l = 0, 1, .... */
static void ssrfb(const double* V, const double* T, double* Ck, double* Ci, int nb, int ib) {
  double w[64];
  for (int l0 = 0; l0 < nb; l0 += ib) {
    const double* Tl = T + (size_t)l0 * ib;
    for (int j = 0; j < nb; ++j) {
      double* ck = Ck + (size_t)j * nb;
      double* ci = Ci + (size_t)j * nb;
      for (int a = 0; a < ib; ++a) {
        const double* va = V + (size_t)(l0 + a) * nb;
        double s = ck[l0 + a];
        for (int r = 0; r < nb; ++r) s += va[r] * ci[r];
        w[a] = s;
      }
      apply_tt(Tl, ib, w);
      for (int a = 0; a < ib; ++a) {
        const double* va = V + (size_t)(l0 + a) * nb;
        ck[l0 + a] -= w[a];
        for (int r = 0; r < nb; ++r) ci[r] -= va[r] * w[a];
      }
    }
  }
}

/* ---- the task DAG (Section 3.3) ------------------------------------------
 * Algorithm 1's tasks in sequential order; each names the data it reads and
 * writes.  A diagonal tile is two regions (its upper triangle with R, its
 * strictly lower part with V), so LARFB(k, j), which reads V_kk, and
 * TSQRT(k, i), which rewrites R_kk, do not wait on each other -- the DAG of
 * the paper's Figure 2.  Edges come from the sequential order: a read waits
 * for the last writer, a write for the last writer and every reader since. */
enum { K_GEQRT = 0, K_TSQRT = 1, K_LARFB = 2, K_SSRFB = 3 }; /* static priority order */

typedef struct {
  int kind, k, i, j;
  int npred;        /* unfinished predecessors */
  int nsucc, csucc; /* successor list */
  int* succ;
} task_t;

typedef struct {
  int writer;     /* last writing task or -1 */
  int nread, cread;
  int* readers;   /* readers since the last write */
} region_t;

static void add_edge(task_t* ts, int from, int to) {
  task_t* f = &ts[from];
  for (int e = 0; e < f->nsucc; ++e)
    if (f->succ[e] == to) return;
  if (f->nsucc == f->csucc) {
    f->csucc = f->csucc ? 2 * f->csucc : 4;
    f->succ = (int*)realloc(f->succ, sizeof(int) * (size_t)f->csucc);
  }
  f->succ[f->nsucc++] = to;
  ts[to].npred++;
}

static void access_region(task_t* ts, region_t* rg, int t, int write) {
  if (rg->writer >= 0 && rg->writer != t) add_edge(ts, rg->writer, t);
  if (write) {
    for (int e = 0; e < rg->nread; ++e)
      if (rg->readers[e] != t) add_edge(ts, rg->readers[e], t);
    rg->writer = t;
    rg->nread = 0;
  } else {
    if (rg->nread == rg->cread) {
      rg->cread = rg->cread ? 2 * rg->cread : 4;
      rg->readers = (int*)realloc(rg->readers, sizeof(int) * (size_t)rg->cread);
    }
    rg->readers[rg->nread++] = t;
  }
}

/* ---- dynamic scheduling ----------------------------------------------------
 * Ready tasks wait in a heap ordered by the paper's static priorities
 * (GEQRT, TSQRT, LARFB, SSRFB; then smaller k, i, j); threads take the best
 * ready task, run it, and release its successors. */
typedef struct {
  grid_t* g;
  task_t* ts;
  int ntasks, done;
  int* heap;
  int nheap;
  pthread_mutex_t mu;
  pthread_cond_t cv;
} sched_t;

static int before(const task_t* a, const task_t* b) {
  if (a->kind != b->kind) return a->kind < b->kind;
  if (a->k != b->k) return a->k < b->k;
  if (a->i != b->i) return a->i < b->i;
  return a->j < b->j;
}

static void heap_push(sched_t* s, int t) {
  int x = s->nheap++;
  s->heap[x] = t;
  while (x > 0) {
    const int up = (x - 1) / 2;
    if (!before(&s->ts[s->heap[x]], &s->ts[s->heap[up]])) break;
    const int tmp = s->heap[x];
    s->heap[x] = s->heap[up];
    s->heap[up] = tmp;
    x = up;
  }
}

static int heap_pop(sched_t* s) {
  const int top = s->heap[0];
  s->heap[0] = s->heap[--s->nheap];
  int x = 0;
  for (;;) {
    const int l = 2 * x + 1, r = l + 1;
    int best = x;
    if (l < s->nheap && before(&s->ts[s->heap[l]], &s->ts[s->heap[best]])) best = l;
    if (r < s->nheap && before(&s->ts[s->heap[r]], &s->ts[s->heap[best]])) best = r;
    if (best == x) break;
    const int tmp = s->heap[x];
    s->heap[x] = s->heap[best];
    s->heap[best] = tmp;
    x = best;
  }
  return top;
}

static void run_task(const grid_t* g, const task_t* t) {
  const int nb = g->nb, ib = g->ib;
  switch (t->kind) {
    case K_GEQRT: geqrt(tile(g, t->k, t->k), tblock(g, t->k, t->k), nb, ib); break;
    case K_LARFB: larfb(tile(g, t->k, t->k), tblock(g, t->k, t->k), tile(g, t->k, t->j), nb, ib); break;
    case K_TSQRT: tsqrt(tile(g, t->k, t->k), tile(g, t->i, t->k), tblock(g, t->i, t->k), nb, ib); break;
    default:
      ssrfb(tile(g, t->i, t->k), tblock(g, t->i, t->k), tile(g, t->k, t->j), tile(g, t->i, t->j), nb, ib);
      break;
  }
}

static void* worker(void* arg) {
  sched_t* s = (sched_t*)arg;
  pthread_mutex_lock(&s->mu);
  while (s->done < s->ntasks) {
    if (s->nheap == 0) {
      pthread_cond_wait(&s->cv, &s->mu);
      continue;
    }
    const int t = heap_pop(s);
    pthread_mutex_unlock(&s->mu);
    run_task(s->g, &s->ts[t]);
    pthread_mutex_lock(&s->mu);
    s->done++;
    const task_t* tt = &s->ts[t];
    for (int e = 0; e < tt->nsucc; ++e)
      if (--s->ts[tt->succ[e]].npred == 0) {
        heap_push(s, tt->succ[e]);
        pthread_cond_signal(&s->cv);
      }
    if (s->done == s->ntasks) pthread_cond_broadcast(&s->cv);
  }
  pthread_mutex_unlock(&s->mu);
  return NULL;
}

/* Tiled QR of the column-major m x n matrix A (lda) with tile nb and inner
 * block ib on `nthreads` threads.  On return A holds R on and above the
 * diagonal and the tiled V below it (as the NumPy oracle's factors), T holds
 * the ib x nb blocks of every (i, k), k < min(p, q), i >= k, at
 * (k p - k (k - 1) / 2 + i - k) ib nb.  *seconds receives the wall time of
 * the task execution (packing excluded).  Returns 0, or -1 for invalid
 * arguments or a failed allocation. */
int ctqr_factor(int m, int n, double* A, int lda, int nb, int ib, double* T, int nthreads, double* seconds) {
  if (m < 1 || n < 1 || lda < m || nb < 1 || ib < 1 || ib > 64 || nb % ib != 0 || nthreads < 1) return -1;
  grid_t g;
  g.nb = nb;
  g.ib = ib;
  g.p = (m + nb - 1) / nb;
  g.q = (n + nb - 1) / nb;
  g.T = T;
  const int kt = g.p < g.q ? g.p : g.q;
  g.tiles = (double*)calloc((size_t)g.p * g.q * nb * nb, sizeof(double));
  if (!g.tiles) return -1;
  for (int c = 0; c < n; ++c)
    for (int r = 0; r < m; ++r) tile(&g, r / nb, c / nb)[(r % nb) + (size_t)(c % nb) * nb] = A[r + (size_t)c * lda];
  /* Algorithm 1 in sequential order */
  long long cnt = 0;
  for (int k = 0; k < kt; ++k) cnt += 1 + (g.q - k - 1) + (long long)(g.p - k - 1) * (1 + (g.q - k - 1));
  task_t* ts = (task_t*)calloc((size_t)cnt, sizeof(task_t));
  const size_t nreg = (size_t)g.p * g.q * 2 + (size_t)g.p * g.q;
  region_t* rg = (region_t*)calloc(nreg, sizeof(region_t));
  int* heap = (int*)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
  if (!ts || !rg || !heap) {
    free(g.tiles); free(ts); free(rg); free(heap);
    return -1;
  }
  for (size_t r = 0; r < nreg; ++r) rg[r].writer = -1;
#define UP(i, j) (&rg[2 * ((size_t)(i) + (size_t)(j) * g.p)])
#define LO(i, j) (&rg[2 * ((size_t)(i) + (size_t)(j) * g.p) + 1])
#define TR(i, k) (&rg[2 * (size_t)g.p * g.q + (size_t)(i) + (size_t)(k) * g.p])
  int nt = 0;
  for (int k = 0; k < kt; ++k) {
    task_t* t = &ts[nt];
    t->kind = K_GEQRT; t->k = k; t->i = k; t->j = k;
    access_region(ts, UP(k, k), nt, 1);
    access_region(ts, LO(k, k), nt, 1);
    access_region(ts, TR(k, k), nt, 1);
    ++nt;
    for (int j = k + 1; j < g.q; ++j) {
      t = &ts[nt];
      t->kind = K_LARFB; t->k = k; t->i = k; t->j = j;
      access_region(ts, LO(k, k), nt, 0);
      access_region(ts, TR(k, k), nt, 0);
      access_region(ts, UP(k, j), nt, 1);
      access_region(ts, LO(k, j), nt, 1);
      ++nt;
    }
    for (int i = k + 1; i < g.p; ++i) {
      t = &ts[nt];
      t->kind = K_TSQRT; t->k = k; t->i = i; t->j = k;
      access_region(ts, UP(k, k), nt, 1);
      access_region(ts, UP(i, k), nt, 1);
      access_region(ts, LO(i, k), nt, 1);
      access_region(ts, TR(i, k), nt, 1);
      const int ts_id = nt++;
      (void)ts_id;
      for (int j = k + 1; j < g.q; ++j) {
        t = &ts[nt];
        t->kind = K_SSRFB; t->k = k; t->i = i; t->j = j;
        access_region(ts, UP(i, k), nt, 0);
        access_region(ts, LO(i, k), nt, 0);
        access_region(ts, TR(i, k), nt, 0);
        access_region(ts, UP(k, j), nt, 1);
        access_region(ts, LO(k, j), nt, 1);
        access_region(ts, UP(i, j), nt, 1);
        access_region(ts, LO(i, j), nt, 1);
        ++nt;
      }
    }
  }
#undef UP
#undef LO
#undef TR
  for (size_t r = 0; r < nreg; ++r) free(rg[r].readers);
  free(rg);
  sched_t s;
  s.g = &g;
  s.ts = ts;
  s.ntasks = nt;
  s.done = 0;
  s.heap = heap;
  s.nheap = 0;
  pthread_mutex_init(&s.mu, NULL);
  pthread_cond_init(&s.cv, NULL);
  for (int t = 0; t < nt; ++t)
    if (ts[t].npred == 0) heap_push(&s, t);
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
  int started = 0;
  for (int a = 0; th && a < nthreads; ++a)
    if (pthread_create(&th[a], NULL, worker, &s) == 0) ++started;
  if (started == 0) worker(&s);
  for (int a = 0; a < started; ++a) pthread_join(th[a], NULL);
  clock_gettime(CLOCK_MONOTONIC, &t1);
  free(th);
  if (seconds) *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
  pthread_mutex_destroy(&s.mu);
  pthread_cond_destroy(&s.cv);
  for (int t = 0; t < nt; ++t) free(ts[t].succ);
  free(ts);
  free(heap);
  for (int c = 0; c < n; ++c)
    for (int r = 0; r < m; ++r) A[r + (size_t)c * lda] = tile(&g, r / nb, c / nb)[(r % nb) + (size_t)(c % nb) * nb];
  free(g.tiles);
  return 0;
}
