/*
 * Plain FP64 CPU oracle for the gravity force path of the AREPO code paper
 * (Weinberger, Springel & Pakmor, "The AREPO public code release").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference legs may load this library.  It shares
 * no code, header, table or helper with the CUDA library; the two meet only
 * through the seeded input generators.
 *
 * Everything here is deliberately plain: double precision throughout, one
 * target particle at a time, no blocking or reordering beyond what each
 * passage defines.  OpenMP parallelises the loop over target particles only.
 *
 * Contents (paper section in brackets):
 *   spline softening kernel of GADGET, Newtonian beyond h = 2.8 eps   [Sec. 3.2]
 *   TreePM short-range factors (Gaussian force split)                [Sec. 3.4]
 *   softened direct summation (exact target, open boundaries)        [Sec. 3]
 *   oct-tree of key prefixes with monopole moments                   [Sec. 3.1]
 *   per-particle tree walk: geometric / relative opening criterion,
 *     1.2 L box guard, short-range cutoff                            [Sec. 3.1, 3.4]
 *   Ewald summation with neutralising background (periodic target)   [Sec. 2.2, 3.1]
 *   Ewald correction of the periodic tree walk (table, trilinear)    [Sec. 3.1]
 *
 * Readings where the paper is silent or garbled are stated at each function.
 * The parity of every function is pinned by the CPU tests (closed forms,
 * quadrature, brute force and invariants); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXLEVEL 21 /* 21 bits per axis -> 63-bit keys (depth-limit reading) */
#define ORC_EWALD_KMAX 64

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Spline softening (Sec. 3.2).                                              */
/* The softened potential of a point mass is that of the cubic-spline (M4)   */
/* density with support h:                                                   */
/*   W(u) = 8/(pi h^3) (1 - 6u^2 + 6u^3)  for 0 <= u < 1/2                   */
/*   W(u) = 8/(pi h^3) 2 (1-u)^3          for 1/2 <= u < 1, zero beyond,     */
/* u = r/h.  With h = 2.8 eps the potential at zero lag is -G m / eps and    */
/* the force is exactly Newtonian for r >= h, as the paper states.           */
/* The force on i from j is a = -G m_j (x_i - x_j) kforce(r); the potential */
/* is G m_j kpot(r).  The polynomials below are the enclosed-mass and        */
/* potential integrals of W (tests check them by quadrature of W).           */
/* ------------------------------------------------------------------------ */
double orc_kforce(double r, double h)
{
    if (r >= h)
        return 1.0 / (r * r * r);
    double u = r / h, h3 = h * h * h;
    if (u < 0.5)
        return (32.0 / 3.0 - 192.0 / 5.0 * u * u + 32.0 * u * u * u) / h3;
    return (64.0 / 3.0 - 48.0 * u + 192.0 / 5.0 * u * u - 32.0 / 3.0 * u * u * u - 1.0 / (15.0 * u * u * u)) / h3;
}

double orc_kpot(double r, double h)
{
    if (r >= h)
        return -1.0 / r;
    double u = r / h, u2 = u * u;
    if (u < 0.5)
        return (16.0 / 3.0 * u2 - 48.0 / 5.0 * u2 * u2 + 32.0 / 5.0 * u2 * u2 * u - 14.0 / 5.0) / h;
    return (32.0 / 3.0 * u2 - 16.0 * u2 * u + 48.0 / 5.0 * u2 * u2 - 32.0 / 15.0 * u2 * u2 * u - 16.0 / 5.0 +
            1.0 / (15.0 * u)) / h;
}

/* ------------------------------------------------------------------------ */
/* TreePM split (Sec. 3.4).  The long-range potential is the k-space         */
/* potential times exp(-k^2 r_s^2), i.e. -G m erf(r / 2 r_s) / r in real     */
/* space.  The short-range remainder multiplies the Newtonian force by       */
/*   g_s(r) = erfc(r / 2 r_s) + r / (sqrt(pi) r_s) exp(-r^2 / 4 r_s^2)       */
/* and the Newtonian potential by erfc(r / 2 r_s).  (The printed factor has  */
/* a sign-flipped exponent and names the complement; this is the reading     */
/* consistent with the printed k-space filter.)  Inside the softening the    */
/* softened kernels are multiplied by the same factors.                      */
/* ------------------------------------------------------------------------ */
double orc_gshort_force(double r, double rs)
{
    double x = r / (2.0 * rs);
    return erfc(x) + r / (sqrt(ORC_PI) * rs) * exp(-x * x);
}

double orc_gshort_pot(double r, double rs)
{
    return erfc(r / (2.0 * rs));
}

/* ------------------------------------------------------------------------ */
/* Softened direct summation, open boundaries: the exact target of the tree */
/* walk (Sec. 3).  a_i = sum_{j != i} -G m_j (x_i - x_j) kforce(r_ij),       */
/* phi_i = sum_{j != i} G m_j kpot(r_ij).                                    */
/* ------------------------------------------------------------------------ */
void orc_direct(int64_t n, const double *pos, const float *mass, int64_t nt, const uint32_t *targets, double G,
                double h, double *acc, double *pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double ax = 0, ay = 0, az = 0, ph = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double m = (double)mass[j];
            double kf = orc_kforce(r, h);
            ax -= m * dx * kf;
            ay -= m * dy * kf;
            az -= m * dz * kf;
            ph += m * orc_kpot(r, h);
        }
        acc[3 * t] = G * ax;
        acc[3 * t + 1] = G * ay;
        acc[3 * t + 2] = G * az;
        pot[t] = G * ph;
    }
}

/* ------------------------------------------------------------------------ */
/* Direct sum with per-particle softening (Sec. 3.2): particles may carry    */
/* different spline supports; a pair interacts with the larger of the two.  */
/* ------------------------------------------------------------------------ */
void orc_direct_soft(int64_t n, const double *pos, const float *mass, const float *hsoft, int64_t nt,
                     const uint32_t *targets, double G, double *acc, double *pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double ax = 0, ay = 0, az = 0, ph = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i)
                continue;
            double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1], dz = pos[3 * i + 2] - pos[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double m = (double)mass[j];
            double h = hsoft[i] > hsoft[j] ? (double)hsoft[i] : (double)hsoft[j];
            double kf = orc_kforce(r, h);
            ax -= m * dx * kf;
            ay -= m * dy * kf;
            az -= m * dz * kf;
            ph += m * orc_kpot(r, h);
        }
        acc[3 * t] = G * ax;
        acc[3 * t + 1] = G * ay;
        acc[3 * t + 2] = G * az;
        pot[t] = G * ph;
    }
}

/* ------------------------------------------------------------------------ */
/* Oct-tree (Sec. 3.1).                                                      */
/*                                                                           */
/* Root.  Open boundaries: a cubical root of power-of-two side L0, the       */
/* smallest with L0 >= 1.25 * (largest extent of the particle set), placed   */
/* at a random offset inside the slack (the paper randomises the placement  */
/* of the tree domain for every construction): x0 = lo - s (L0 - ext_a),     */
/* rounded down to the 2^-21 L0 grid, with s in [0, 1) passed in.           */
/* Periodic: the whole box is shifted by s * box and wrapped, x0 = 0,        */
/* L0 = box (the paper's random box shift).                                   */
/*                                                                           */
/* Node set.  The paper inserts particles one by one and splits every leaf   */
/* that would hold two particles.  The resulting set of non-empty cells does */
/* not depend on the insertion order: a cell at level l+1 exists exactly     */
/* when its parent holds more than one particle.  With a leaf bucket B the   */
/* same rule reads "more than B"; B = 1 is the paper's tree.  The depth is   */
/* capped at level 21 (the paper caps at 30 and scatters coincident          */
/* particles randomly; here a level-21 cell simply keeps all of them).       */
/* The cells are found from integer cell coordinates q = floor((x - x0) /    */
/* (L0 / 2^21)): the level-l cell of a particle is q >> (21 - l).  Children  */
/* are visited in ascending octant order (x bit 0, y bit 1, z bit 2) and     */
/* particles in ascending (key, index) order, where the key interleaves the  */
/* q bits -- the Morton order the paper uses for its domain chunks.          */
/*                                                                           */
/* Monopoles.  Node mass M = sum of child masses and S = sum of child        */
/* m x in ascending octant order (a leaf sums its particles in order);       */
/* centre of mass = S / M, all in FP64.                                      */
/* ------------------------------------------------------------------------ */
typedef struct orc_tree {
    int64_t n;
    int periodic;
    double box;
    double x0[3], L0;
    int bucket;
    double *x;       /* positions used by the tree (shifted / wrapped if periodic), original order */
    const float *m;  /* caller's masses, original order */
    uint64_t *key;   /* sorted */
    uint32_t *perm;  /* sorted position -> original index */
    uint32_t *rank;  /* original index -> sorted position */
    int64_t nnodes, cap;
    uint8_t *level;
    uint64_t *prefix;
    uint32_t *first, *count, *skip;
    double *mass, *com; /* com: 3 per node */
    const float *hsoft; /* per-particle spline support (original order), NULL: uniform */
    double *hmax, *hmin; /* per node: largest and smallest support of its particles */
} orc_tree;

static uint64_t orc_spread(uint64_t v)
{
    /* place bit b of v at bit 3b (v < 2^21) */
    uint64_t out = 0;
    for (int b = 0; b < ORC_MAXLEVEL; b++)
        out |= ((v >> b) & 1ull) << (3 * b);
    return out;
}

static double orc_pow2_ceil(double x)
{
    int e;
    double f = frexp(x, &e); /* x = f 2^e, f in [0.5, 1) */
    return (f == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

static int orc_cmp_pair(const void *a, const void *b)
{
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    if (x[0] != y[0])
        return x[0] < y[0] ? -1 : 1;
    if (x[1] != y[1])
        return x[1] < y[1] ? -1 : 1;
    return 0;
}

static int64_t orc_new_node(orc_tree *t)
{
    if (t->nnodes == t->cap) {
        int64_t c = t->cap ? 2 * t->cap : 1024;
        t->level = realloc(t->level, c * sizeof(uint8_t));
        t->prefix = realloc(t->prefix, c * sizeof(uint64_t));
        t->first = realloc(t->first, c * sizeof(uint32_t));
        t->count = realloc(t->count, c * sizeof(uint32_t));
        t->skip = realloc(t->skip, c * sizeof(uint32_t));
        t->mass = realloc(t->mass, c * sizeof(double));
        t->com = realloc(t->com, 3 * c * sizeof(double));
        t->cap = c;
    }
    return t->nnodes++;
}

/* Builds the subtree of cell (level, prefix) holding sorted particles [lo, hi);
 * returns its total mass and mass-weighted position sum S. */
static void orc_build_node(orc_tree *t, int level, uint64_t prefix, int64_t lo, int64_t hi, double *Mout, double S[3])
{
    int64_t id = orc_new_node(t);
    t->level[id] = (uint8_t)level;
    t->prefix[id] = prefix;
    t->first[id] = (uint32_t)lo;
    t->count[id] = (uint32_t)(hi - lo);
    double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    if (hi - lo > t->bucket && level < ORC_MAXLEVEL) {
        int shift = 3 * (ORC_MAXLEVEL - level - 1);
        int64_t a = lo;
        for (int oct = 0; oct < 8; oct++) {
            int64_t b = a;
            while (b < hi && (int)((t->key[b] >> shift) & 7ull) == oct)
                b++;
            if (b > a) {
                double Mc, Sc[3];
                orc_build_node(t, level + 1, (prefix << 3) | (uint64_t)oct, a, b, &Mc, Sc);
                M += Mc;
                sx += Sc[0];
                sy += Sc[1];
                sz += Sc[2];
            }
            a = b;
        }
    } else {
        for (int64_t s = lo; s < hi; s++) {
            uint32_t j = t->perm[s];
            double m = (double)t->m[j];
            M += m;
            sx += m * t->x[3 * j];
            sy += m * t->x[3 * j + 1];
            sz += m * t->x[3 * j + 2];
        }
    }
    t->mass[id] = M;
    t->com[3 * id] = sx / M;
    t->com[3 * id + 1] = sy / M;
    t->com[3 * id + 2] = sz / M;
    t->skip[id] = (uint32_t)t->nnodes; /* first node after this subtree (pre-order) */
    *Mout = M;
    S[0] = sx;
    S[1] = sy;
    S[2] = sz;
}

void orc_tree_free(orc_tree *t)
{
    if (!t)
        return;
    free(t->x);
    free(t->key);
    free(t->perm);
    free(t->rank);
    free(t->level);
    free(t->prefix);
    free(t->first);
    free(t->count);
    free(t->skip);
    free(t->mass);
    free(t->com);
    free(t->hmax);
    free(t->hmin);
    free(t);
}

orc_tree *orc_tree_build(int64_t n, const double *pos, const float *mass, int periodic, double box,
                         const double shift[3], int bucket)
{
    if (n <= 0 || bucket < 1)
        return NULL;
    orc_tree *t = calloc(1, sizeof(orc_tree));
    t->n = n;
    t->periodic = periodic;
    t->box = box;
    t->bucket = bucket;
    t->m = mass;
    t->x = malloc(3 * n * sizeof(double));
    if (periodic) {
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < 3; a++) {
                double v = pos[3 * i + a] + shift[a] * box;
                if (v >= box)
                    v -= box;
                t->x[3 * i + a] = v;
            }
        t->x0[0] = t->x0[1] = t->x0[2] = 0.0;
        t->L0 = box;
    } else {
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++)
            lo[a] = hi[a] = pos[a];
        for (int64_t i = 0; i < n; i++)
            for (int a = 0; a < 3; a++) {
                double v = pos[3 * i + a];
                t->x[3 * i + a] = v;
                if (v < lo[a])
                    lo[a] = v;
                if (v > hi[a])
                    hi[a] = v;
            }
        double ext = 0.0;
        for (int a = 0; a < 3; a++)
            if (hi[a] - lo[a] > ext)
                ext = hi[a] - lo[a];
        if (!(ext > 0.0))
            ext = 1.0;
        double L0 = orc_pow2_ceil(1.25 * ext);
        double unit = ldexp(L0, -ORC_MAXLEVEL);
        for (int a = 0; a < 3; a++) {
            double slack = L0 - (hi[a] - lo[a]);
            double x0 = lo[a] - shift[a] * slack;
            t->x0[a] = floor(x0 / unit) * unit;
        }
        t->L0 = L0;
    }
    /* keys, then a stable sort by (key, original index) */
    double scale = ldexp(1.0, ORC_MAXLEVEL) / t->L0;
    uint64_t *pairs = malloc(2 * n * sizeof(uint64_t));
    for (int64_t i = 0; i < n; i++) {
        uint64_t k = 0;
        for (int a = 0; a < 3; a++) {
            double f = floor((t->x[3 * i + a] - t->x0[a]) * scale);
            int64_t q = (int64_t)f;
            if (f < 0.0)
                q = 0;
            if (f > (double)((1 << ORC_MAXLEVEL) - 1))
                q = (1 << ORC_MAXLEVEL) - 1;
            k |= orc_spread((uint64_t)q) << a;
        }
        pairs[2 * i] = k;
        pairs[2 * i + 1] = (uint64_t)i;
    }
    qsort(pairs, n, 2 * sizeof(uint64_t), orc_cmp_pair);
    t->key = malloc(n * sizeof(uint64_t));
    t->perm = malloc(n * sizeof(uint32_t));
    t->rank = malloc(n * sizeof(uint32_t));
    for (int64_t s = 0; s < n; s++) {
        t->key[s] = pairs[2 * s];
        t->perm[s] = (uint32_t)pairs[2 * s + 1];
        t->rank[t->perm[s]] = (uint32_t)s;
    }
    free(pairs);
    double M, S[3];
    orc_build_node(t, 0, 0, 0, n, &M, S);
    return t;
}

int64_t orc_tree_nnodes(const orc_tree *t) { return t->nnodes; }

/* Per-particle softening (Sec. 3.2) for the walk: each node records the      */
/* largest and smallest support among its particles.  hsoft (original order) */
/* must outlive the tree; NULL returns to the uniform softening.             */
void orc_tree_set_soft(orc_tree *t, const float *hsoft)
{
    free(t->hmax);
    free(t->hmin);
    t->hmax = t->hmin = NULL;
    t->hsoft = hsoft;
    if (!hsoft)
        return;
    t->hmax = malloc(t->nnodes * sizeof(double));
    t->hmin = malloc(t->nnodes * sizeof(double));
    for (int64_t id = 0; id < t->nnodes; id++) {
        double hi = 0.0, lo = INFINITY;
        for (uint32_t s = t->first[id]; s < t->first[id] + t->count[id]; s++) {
            double h = hsoft[t->perm[s]];
            if (h > hi)
                hi = h;
            if (h < lo)
                lo = h;
        }
        t->hmax[id] = hi;
        t->hmin[id] = lo;
    }
}

void orc_tree_root(const orc_tree *t, double x0[3], double *L0)
{
    x0[0] = t->x0[0];
    x0[1] = t->x0[1];
    x0[2] = t->x0[2];
    *L0 = t->L0;
}

void orc_tree_export(const orc_tree *t, uint64_t *key, uint32_t *perm, uint8_t *level, uint64_t *prefix,
                     uint32_t *first, uint32_t *count, uint32_t *skip, double *mass, double *com, double *xtree)
{
    if (key) memcpy(key, t->key, t->n * sizeof(uint64_t));
    if (perm) memcpy(perm, t->perm, t->n * sizeof(uint32_t));
    if (level) memcpy(level, t->level, t->nnodes * sizeof(uint8_t));
    if (prefix) memcpy(prefix, t->prefix, t->nnodes * sizeof(uint64_t));
    if (first) memcpy(first, t->first, t->nnodes * sizeof(uint32_t));
    if (count) memcpy(count, t->count, t->nnodes * sizeof(uint32_t));
    if (skip) memcpy(skip, t->skip, t->nnodes * sizeof(uint32_t));
    if (mass) memcpy(mass, t->mass, t->nnodes * sizeof(double));
    if (com) memcpy(com, t->com, 3 * t->nnodes * sizeof(double));
    if (xtree) memcpy(xtree, t->x, 3 * t->n * sizeof(double));
}

/* Geometric centre and side length of node id, from (level, prefix). */
static void orc_node_geometry(const orc_tree *t, int64_t id, double c[3], double *L)
{
    int level = t->level[id];
    uint64_t p = t->prefix[id];
    double side = ldexp(t->L0, -level);
    for (int a = 0; a < 3; a++) {
        uint64_t ia = 0;
        for (int b = 0; b < level; b++)
            ia |= ((p >> (3 * b + a)) & 1ull) << b;
        c[a] = t->x0[a] + ((double)ia + 0.5) * side;
    }
    *L = side;
}

/* ------------------------------------------------------------------------ */
/* Tree walk (Sec. 3.1, 3.4).  For each target i, from the root:             */
/*  - TreePM: a node whose cube lies farther than r_cut = a_cut r_s from the */
/*    particle (minimum distance, periodic minimum image) is ignored;        */
/*  - otherwise the node is opened when the particle lies inside the cube of */
/*    side 1.2 L centred on the node's geometric centre (box guard), or when */
/*    the opening criterion holds: geometric  L > theta d, or relative       */
/*    G M L^2 / d^4 > alpha |a_old|, d = distance to the centre of mass;    */
/*  - an opened internal node hands over to its children (ascending octant), */
/*    an opened leaf interacts particle by particle (j != i; TreePM: only    */
/*    pairs closer than r_cut), and an unopened node adds its monopole.      */
/* Pair law: spline-softened, times the short-range factors under TreePM.    */
/* Every monopole and pair term counts as one interaction.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double G, h;
    int crit;          /* 0 geometric (Barnes-Hut), 1 relative */
    double theta;      /* ErrTolTheta */
    double alpha;      /* ErrTolForceAcc */
    int box_guard;     /* 1: apply the 1.2 L box rule */
    int treepm;        /* 1: short-range force only, with cutoff */
    double rs, rcut;   /* split scale r_s and cutoff radius a_cut r_s */
    int ewald;         /* 1 (periodic tree, treepm = 0): add the Ewald correction */
    const double *etab; /* correction table of orc_ewald_table, (ent+1)^3 x 4 */
    int ent;           /* table intervals per axis over [0, box/2] */
} orc_walk_params;

static void orc_ewald_lookup(const orc_walk_params *p, double box, double dx, double dy, double dz, double f[3],
                             double *phi);

static inline double orc_wrap(double d, int periodic, double box)
{
    if (!periodic)
        return d;
    if (d > 0.5 * box)
        d -= box;
    else if (d < -0.5 * box)
        d += box;
    return d;
}

static inline void orc_pair(const orc_walk_params *p, double h, double dx, double dy, double dz, double m,
                            double acc[3], double *pot)
{
    /* (dx,dy,dz) = x_source - x_target; h the spline support of the pair */
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double kf = orc_kforce(r, h), kp = orc_kpot(r, h);
    if (p->treepm) {
        kf *= orc_gshort_force(r, p->rs);
        kp *= orc_gshort_pot(r, p->rs);
    }
    acc[0] += m * dx * kf;
    acc[1] += m * dy * kf;
    acc[2] += m * dz * kf;
    *pot += m * kp;
}

/* Monopole / pair term of the periodic tree without the mesh: the nearest
 * image (spline-softened) plus the Ewald correction at the same separation. */
static inline void orc_pair_ewald(const orc_walk_params *p, double h, double box, double dx, double dy, double dz,
                                  double m, double acc[3], double *pot)
{
    orc_pair(p, h, dx, dy, dz, m, acc, pot);
    double f[3], ph;
    orc_ewald_lookup(p, box, dx, dy, dz, f, &ph);
    acc[0] += m * f[0];
    acc[1] += m * f[1];
    acc[2] += m * f[2];
    *pot += m * ph;
}

static void orc_walk_one(const orc_tree *t, int64_t i, double aold, const orc_walk_params *p, double acc[3],
                         double *pot, uint32_t *nint)
{
    const double *xi = &t->x[3 * i];
    double box = t->box;
    int per = t->periodic;
    double rcut2 = p->rcut * p->rcut;
    uint32_t self = t->rank[i];
    const double hi = t->hsoft ? (double)t->hsoft[i] : p->h; /* the target's support */
    acc[0] = acc[1] = acc[2] = 0.0;
    *pot = 0.0;
    uint32_t cnt = 0;
    /* iterative depth-first traversal of the pre-order node array: after a
     * node, either descend to its first child (the next node) or jump past its
     * subtree (skip) */
    int64_t id = 0;
    while (id < t->nnodes) {
        double c[3], L;
        orc_node_geometry(t, id, c, &L);
        double px = orc_wrap(xi[0] - c[0], per, box), py = orc_wrap(xi[1] - c[1], per, box),
               pz = orc_wrap(xi[2] - c[2], per, box);
        if (p->treepm) {
            double ex = fabs(px) - 0.5 * L, ey = fabs(py) - 0.5 * L, ez = fabs(pz) - 0.5 * L;
            ex = ex > 0 ? ex : 0;
            ey = ey > 0 ? ey : 0;
            ez = ez > 0 ? ez : 0;
            if (ex * ex + ey * ey + ez * ez > rcut2) {
                id = t->skip[id];
                continue;
            }
        }
        double dx = orc_wrap(t->com[3 * id] - xi[0], per, box), dy = orc_wrap(t->com[3 * id + 1] - xi[1], per, box),
               dz = orc_wrap(t->com[3 * id + 2] - xi[2], per, box);
        double d2 = dx * dx + dy * dy + dz * dz;
        int open = 0;
        if (p->box_guard && fabs(px) <= 0.6 * L && fabs(py) <= 0.6 * L && fabs(pz) <= 0.6 * L)
            open = 1;
        /* Sec. 3.2: a node of mixed softenings whose largest exceeds the
         * target's, closer than that largest, is always opened */
        double hnode = hi;
        if (t->hsoft) {
            if (t->hmin[id] < t->hmax[id] && hi < t->hmax[id] && d2 < t->hmax[id] * t->hmax[id])
                open = 1;
            hnode = hi > t->hmax[id] ? hi : t->hmax[id];
        }
        if (!open) {
            if (p->crit == 0)
                open = L * L > p->theta * p->theta * d2;
            else
                open = p->G * t->mass[id] * L * L > p->alpha * aold * d2 * d2;
        }
        int leaf = (t->skip[id] == id + 1);
        int ew = per && p->ewald && !p->treepm;
        if (!open) {
            if (ew)
                orc_pair_ewald(p, hnode, box, dx, dy, dz, t->mass[id], acc, pot);
            else
                orc_pair(p, hnode, dx, dy, dz, t->mass[id], acc, pot);
            cnt++;
            id = t->skip[id];
        } else if (!leaf) {
            id = id + 1;
        } else {
            for (uint32_t s = t->first[id]; s < t->first[id] + t->count[id]; s++) {
                if (s == self)
                    continue;
                uint32_t j = t->perm[s];
                double qx = orc_wrap(t->x[3 * j] - xi[0], per, box), qy = orc_wrap(t->x[3 * j + 1] - xi[1], per, box),
                       qz = orc_wrap(t->x[3 * j + 2] - xi[2], per, box);
                if (p->treepm && qx * qx + qy * qy + qz * qz > rcut2)
                    continue;
                double hp = hi;
                if (t->hsoft && (double)t->hsoft[j] > hp)
                    hp = (double)t->hsoft[j];
                if (ew)
                    orc_pair_ewald(p, hp, box, qx, qy, qz, (double)t->m[j], acc, pot);
                else
                    orc_pair(p, hp, qx, qy, qz, (double)t->m[j], acc, pot);
                cnt++;
            }
            id = t->skip[id];
        }
    }
    if (per && p->ewald && !p->treepm) { /* the particle's own images and background */
        double f[3], ph;
        orc_ewald_lookup(p, box, 0.0, 0.0, 0.0, f, &ph);
        *pot += (double)t->m[i] * ph;
    }
    acc[0] *= p->G;
    acc[1] *= p->G;
    acc[2] *= p->G;
    *pot *= p->G;
    *nint = cnt;
}

void orc_tree_walk(const orc_tree *t, int64_t nt, const uint32_t *targets, const float *a_old,
                   const orc_walk_params *p, double *acc, double *pot, uint32_t *nint, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < nt; k++) {
        double a3[3], ph;
        uint32_t c;
        double aold = a_old ? (double)a_old[k] : 0.0;
        orc_walk_one(t, targets[k], aold, p, a3, &ph, &c);
        acc[3 * k] = a3[0];
        acc[3 * k + 1] = a3[1];
        acc[3 * k + 2] = a3[2];
        pot[k] = ph;
        if (nint)
            nint[k] = c;
    }
}

/* ------------------------------------------------------------------------ */
/* Ewald summation (periodic target, Sec. 2.2 and 3.1).  Poisson's equation */
/* with the mean density subtracted, in a cube of side L (volume V).  With  */
/* the splitting parameter a (alpha_E):                                      */
/*   a_i = -G sum_{j != i} m_j r/r^3 [erfc(a r) + 2 a r/sqrt(pi) e^{-a^2r^2}] */
/*         (minimum image, r < r_E <= L/2)                                   */
/*       - G (4 pi / V) sum_{k != 0} k/k^2 e^{-k^2/4a^2} Im(e^{i k x_i} S(k)) */
/*   S(k) = sum_j m_j e^{-i k x_j},  r = x_i - x_j.                          */
/* The potential is the alpha-independent one of particle i in the lattice  */
/* of all images (own images included, background included):               */
/*   phi_i = -G [ sum_{j != i} m_j erfc(a r)/r                               */
/*          + (4 pi / V) sum_k e^{-k^2/4a^2}/k^2 Re(e^{i k x_i} S(k))        */
/*          - pi M_tot / (a^2 V) - 2 a m_i / sqrt(pi) ].                     */
/* The k sum runs over |n| <= kmax (k = 2 pi n / L), half space doubled.     */
/* The real-space sum uses a cell list; r_E must not exceed L/2.             */
/* ------------------------------------------------------------------------ */
void orc_ewald(int64_t n, const double *pos, const float *mass, int64_t nt, const uint32_t *targets, double G,
               double box, double alpha, double rreal, int kmax, double *acc, double *pot, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
    int nth = omp_get_max_threads();
#else
    int nth = 1;
#endif
    if (kmax < 1 || kmax > ORC_EWALD_KMAX || !(rreal > 0.0) || rreal > 0.5 * box)
        return;
    double V = box * box * box;
    double Mtot = 0.0;
    for (int64_t j = 0; j < n; j++)
        Mtot += (double)mass[j];
    /* half-space k vectors grouped in (nx, ny) columns with a run of nz */
    int K = kmax, W = 2 * K + 1;
    int ncol = 0;
    int *colx = malloc(W * W * sizeof(int)), *coly = malloc(W * W * sizeof(int));
    int *czlo = malloc(W * W * sizeof(int)), *czhi = malloc(W * W * sizeof(int)), *coff = malloc(W * W * sizeof(int));
    int nk = 0;
    for (int nx = 0; nx <= K; nx++)
        for (int ny = -K; ny <= K; ny++) {
            int lo = 1000000, hi = -1000000;
            for (int nz = -K; nz <= K; nz++) {
                int half = (nx > 0) || (nx == 0 && ny > 0) || (nx == 0 && ny == 0 && nz > 0);
                if (!half || nx * nx + ny * ny + nz * nz > K * K)
                    continue;
                if (nz < lo) lo = nz;
                if (nz > hi) hi = nz;
            }
            if (hi < lo)
                continue;
            colx[ncol] = nx;
            coly[ncol] = ny;
            czlo[ncol] = lo;
            czhi[ncol] = hi;
            coff[ncol] = nk;
            nk += hi - lo + 1;
            ncol++;
        }
    double *Sre = calloc((size_t)nk * nth, sizeof(double)), *Sim = calloc((size_t)nk * nth, sizeof(double));
    double tw = 2.0 * ORC_PI / box;
#pragma omp parallel
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double *sr = Sre + (size_t)tid * nk, *si = Sim + (size_t)tid * nk;
        double *er = malloc(3 * W * sizeof(double)), *ei = malloc(3 * W * sizeof(double));
#pragma omp for schedule(static)
        for (int64_t j = 0; j < n; j++) {
            double m = (double)mass[j];
            for (int a = 0; a < 3; a++) {
                /* e^{-i n k1 x} for n = -K..K */
                double c1 = cos(tw * pos[3 * j + a]), s1 = -sin(tw * pos[3 * j + a]);
                double *pr = er + a * W + K, *pi = ei + a * W + K;
                pr[0] = 1.0;
                pi[0] = 0.0;
                for (int q = 1; q <= K; q++) {
                    pr[q] = pr[q - 1] * c1 - pi[q - 1] * s1;
                    pi[q] = pr[q - 1] * s1 + pi[q - 1] * c1;
                    pr[-q] = pr[q];
                    pi[-q] = -pi[q];
                }
            }
            for (int c = 0; c < ncol; c++) {
                double xr = er[colx[c] + K], xi = ei[colx[c] + K];
                double yr = er[W + coly[c] + K], yi = ei[W + coly[c] + K];
                double ar = m * (xr * yr - xi * yi), ai = m * (xr * yi + xi * yr);
                int o = coff[c] - czlo[c];
                for (int nz = czlo[c]; nz <= czhi[c]; nz++) {
                    double zr = er[2 * W + nz + K], zi = ei[2 * W + nz + K];
                    sr[o + nz] += ar * zr - ai * zi;
                    si[o + nz] += ar * zi + ai * zr;
                }
            }
        }
        free(er);
        free(ei);
    }
    for (int t = 1; t < nth; t++)
        for (int k = 0; k < nk; k++) {
            Sre[k] += Sre[(size_t)t * nk + k];
            Sim[k] += Sim[(size_t)t * nk + k];
        }
    /* cell list for the real-space sum */
    int nc = (int)floor(box / (0.5 * rreal));
    if (nc < 1)
        nc = 1;
    if (nc > 256)
        nc = 256;
    double csz = box / nc;
    int span = (int)ceil(rreal / csz);
    if (2 * span + 1 > nc)
        span = -1; /* small box: loop over all particles */
    int64_t ncell = (int64_t)nc * nc * nc;
    int64_t *cstart = calloc(ncell + 1, sizeof(int64_t));
    int64_t *clist = malloc(n * sizeof(int64_t));
    int64_t *cid = malloc(n * sizeof(int64_t));
    for (int64_t j = 0; j < n; j++) {
        int64_t ci[3];
        for (int a = 0; a < 3; a++) {
            double v = pos[3 * j + a] - box * floor(pos[3 * j + a] / box);
            int64_t q = (int64_t)floor(v / csz);
            if (q >= nc) q = nc - 1;
            if (q < 0) q = 0;
            ci[a] = q;
        }
        cid[j] = (ci[0] * nc + ci[1]) * nc + ci[2];
        cstart[cid[j] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++)
        cstart[c + 1] += cstart[c];
    {
        int64_t *fill = malloc(ncell * sizeof(int64_t));
        memcpy(fill, cstart, ncell * sizeof(int64_t));
        for (int64_t j = 0; j < n; j++)
            clist[fill[cid[j]]++] = j;
        free(fill);
    }
    double rr2 = rreal * rreal, a2 = alpha * alpha, sqpi = sqrt(ORC_PI);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = targets[t];
        double xi[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        double ax = 0, ay = 0, az = 0, ph = 0;
        /* real space */
        int64_t lo_c = span < 0 ? 0 : -span, hi_c = span < 0 ? 0 : span;
        int64_t ci[3];
        for (int a = 0; a < 3; a++) {
            double v = xi[a] - box * floor(xi[a] / box);
            ci[a] = (int64_t)floor(v / csz);
            if (ci[a] >= nc) ci[a] = nc - 1;
        }
        for (int64_t ox = lo_c; ox <= hi_c; ox++)
            for (int64_t oy = lo_c; oy <= hi_c; oy++)
                for (int64_t oz = lo_c; oz <= hi_c; oz++) {
                    int64_t j0, j1;
                    if (span < 0) {
                        j0 = 0;
                        j1 = n;
                    } else {
                        int64_t cx = ((ci[0] + ox) % nc + nc) % nc, cy = ((ci[1] + oy) % nc + nc) % nc,
                                cz = ((ci[2] + oz) % nc + nc) % nc;
                        int64_t c = (cx * nc + cy) * nc + cz;
                        j0 = cstart[c];
                        j1 = cstart[c + 1];
                    }
                    for (int64_t q = j0; q < j1; q++) {
                        int64_t j = span < 0 ? q : clist[q];
                        if (j == i)
                            continue;
                        double dx = orc_wrap(xi[0] - pos[3 * j], 1, box), dy = orc_wrap(xi[1] - pos[3 * j + 1], 1, box),
                               dz = orc_wrap(xi[2] - pos[3 * j + 2], 1, box);
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 >= rr2)
                            continue;
                        double r = sqrt(r2), m = (double)mass[j];
                        double ec = erfc(alpha * r);
                        double f = m * (ec + 2.0 * alpha * r / sqpi * exp(-a2 * r2)) / (r2 * r);
                        ax -= f * dx;
                        ay -= f * dy;
                        az -= f * dz;
                        ph -= m * ec / r;
                    }
                }
        /* k space */
        double *pr[3], *pi[3];
        double bufr[3][2 * ORC_EWALD_KMAX + 1], bufi[3][2 * ORC_EWALD_KMAX + 1];
        for (int a = 0; a < 3; a++) {
            double c1 = cos(tw * xi[a]), s1 = sin(tw * xi[a]); /* e^{+i k1 x} */
            pr[a] = bufr[a] + ORC_EWALD_KMAX;
            pi[a] = bufi[a] + ORC_EWALD_KMAX;
            pr[a][0] = 1.0;
            pi[a][0] = 0.0;
            for (int q = 1; q <= K; q++) {
                pr[a][q] = pr[a][q - 1] * c1 - pi[a][q - 1] * s1;
                pi[a][q] = pr[a][q - 1] * s1 + pi[a][q - 1] * c1;
                pr[a][-q] = pr[a][q];
                pi[a][-q] = -pi[a][q];
            }
        }
        double kx_sum = 0, ky_sum = 0, kz_sum = 0, kp_sum = 0;
        for (int c = 0; c < ncol; c++) {
            int nx = colx[c], ny = coly[c];
            double xr = pr[0][nx], xim = pi[0][nx], yr = pr[1][ny], yim = pi[1][ny];
            double br = xr * yr - xim * yim, bi = xr * yim + xim * yr;
            int o = coff[c] - czlo[c];
            for (int nz = czlo[c]; nz <= czhi[c]; nz++) {
                double zr = pr[2][nz], zim = pi[2][nz];
                double er_ = br * zr - bi * zim, ei_ = br * zim + bi * zr; /* e^{i k x_i} */
                double sre = Sre[o + nz], sim = Sim[o + nz];
                double re = er_ * sre - ei_ * sim, im = er_ * sim + ei_ * sre;
                double k2 = tw * tw * (double)(nx * nx + ny * ny + nz * nz);
                double g = exp(-k2 / (4.0 * a2)) / k2;
                kx_sum += g * tw * nx * im;
                ky_sum += g * tw * ny * im;
                kz_sum += g * tw * nz * im;
                kp_sum += g * re;
            }
        }
        double pref = 4.0 * ORC_PI / V * 2.0; /* factor 2: the other half space */
        ax -= pref * kx_sum;
        ay -= pref * ky_sum;
        az -= pref * kz_sum;
        ph -= pref * kp_sum;
        ph += ORC_PI * Mtot / (a2 * V) + 2.0 * alpha * (double)mass[i] / sqpi;
        acc[3 * t] = G * ax;
        acc[3 * t + 1] = G * ay;
        acc[3 * t + 2] = G * az;
        pot[t] = G * ph;
    }
    free(cstart);
    free(clist);
    free(cid);
    free(Sre);
    free(Sim);
    free(colx);
    free(coly);
    free(czlo);
    free(czhi);
    free(coff);
}

/* ------------------------------------------------------------------------ */
/* Ewald correction of the periodic tree (Sec. 3.1: the contributions of the */
/* mirrored images, by the Ewald technique).  For a unit mass (G = 1) at     */
/* separation d = x_source - x_target (nearest image), in a cube of side L  */
/* with the mean density subtracted, the periodic acceleration of the target */
/* is, with the split a = 2 / L,                                             */
/*   a_E(d) = sum_n (d + nL)/s^3 [erfc(a s) + 2 a s/sqrt(pi) e^{-a^2 s^2}]   */
/*            + (4 pi / V) sum_{k != 0} k/k^2 e^{-k^2/4a^2} sin(k.d),        */
/*   s = |d + nL|, k = 2 pi m / L,                                           */
/* and its potential                                                         */
/*   phi_E(d) = -sum_n erfc(a s)/s - (4 pi / V) sum_k e^{-k^2/4a^2}/k^2     */
/*              cos(k.d) + pi / (a^2 V).                                     */
/* The correction is what the nearest image misses: a_E - d/|d|^3 and       */
/* phi_E + 1/|d|; at d = 0 the force correction vanishes and the potential  */
/* correction is the particle's own lattice term (the limit of the n = 0     */
/* real-space term is -2a/sqrt(pi)).  Images |n| <= 4 and |m| <= 5 (both    */
/* sums converged far below FP64 rounding at a = 2 / L).                     */
/* ------------------------------------------------------------------------ */
void orc_ewald_correction(double box, double dx, double dy, double dz, double out[4])
{
    double a = 2.0 / box, a2 = a * a, V = box * box * box, sqpi = sqrt(ORC_PI);
    double f[3] = {0, 0, 0}, ph = 0.0;
    double d2 = dx * dx + dy * dy + dz * dz;
    for (int nx = -4; nx <= 4; nx++)
        for (int ny = -4; ny <= 4; ny++)
            for (int nz = -4; nz <= 4; nz++) {
                double sx = dx + nx * box, sy = dy + ny * box, sz = dz + nz * box;
                double s2 = sx * sx + sy * sy + sz * sz;
                if (nx == 0 && ny == 0 && nz == 0) {
                    if (d2 == 0.0) {
                        ph += 2.0 * a / sqpi; /* lim_{s->0} erf(a s) / s */
                        continue;
                    }
                    double s = sqrt(s2);
                    /* n = 0: only the erfc part differs from the nearest image */
                    double g = erfc(a * s) + 2.0 * a * s / sqpi * exp(-a2 * s2);
                    f[0] += sx / (s2 * s) * (g - 1.0);
                    f[1] += sy / (s2 * s) * (g - 1.0);
                    f[2] += sz / (s2 * s) * (g - 1.0);
                    ph += -erfc(a * s) / s + 1.0 / s;
                    continue;
                }
                double s = sqrt(s2);
                double g = erfc(a * s) + 2.0 * a * s / sqpi * exp(-a2 * s2);
                f[0] += sx / (s2 * s) * g;
                f[1] += sy / (s2 * s) * g;
                f[2] += sz / (s2 * s) * g;
                ph += -erfc(a * s) / s;
            }
    double tw = 2.0 * ORC_PI / box;
    for (int mx = -5; mx <= 5; mx++)
        for (int my = -5; my <= 5; my++)
            for (int mz = -5; mz <= 5; mz++) {
                int m2 = mx * mx + my * my + mz * mz;
                if (m2 == 0 || m2 > 30)
                    continue;
                double kx = tw * mx, ky = tw * my, kz = tw * mz, k2 = tw * tw * m2;
                double w = exp(-k2 / (4.0 * a2)) / k2;
                double kd = kx * dx + ky * dy + kz * dz;
                f[0] += 4.0 * ORC_PI / V * w * kx * sin(kd);
                f[1] += 4.0 * ORC_PI / V * w * ky * sin(kd);
                f[2] += 4.0 * ORC_PI / V * w * kz * sin(kd);
                ph -= 4.0 * ORC_PI / V * w * cos(kd);
            }
    ph += ORC_PI / (a2 * V);
    out[0] = f[0];
    out[1] = f[1];
    out[2] = f[2];
    out[3] = ph;
}

/* The correction on the grid d = (i, j, k) box / (2 nt), 0 <= i, j, k <= nt,
 * as (fx, fy, fz, phi) per point, x slowest. */
void orc_ewald_table(double box, int nt, double *tab, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#endif
    int64_t m = nt + 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < m * m * m; e++) {
        int64_t i = e / (m * m), j = (e / m) % m, k = e % m;
        double step = 0.5 * box / nt;
        orc_ewald_correction(box, i * step, j * step, k * step, &tab[4 * e]);
    }
}

/* Trilinear interpolation of the table at d, folded into [0, box/2]^3: the
 * force correction is odd in its own component and even in the others, the
 * potential correction even in all. */
static void orc_ewald_lookup(const orc_walk_params *p, double box, double dx, double dy, double dz, double f[3],
                             double *phi)
{
    double d[3] = {dx, dy, dz}, sg[3], u[3];
    int i0[3];
    int nt = p->ent;
    for (int a = 0; a < 3; a++) {
        sg[a] = d[a] < 0.0 ? -1.0 : 1.0;
        double t = fabs(d[a]) * (2.0 * nt / box);
        int q = (int)floor(t);
        if (q >= nt)
            q = nt - 1;
        i0[a] = q;
        u[a] = t - q;
    }
    int64_t m = nt + 1;
    double v[4] = {0, 0, 0, 0};
    for (int c = 0; c < 8; c++) {
        int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
        double w = (bx ? u[0] : 1.0 - u[0]) * (by ? u[1] : 1.0 - u[1]) * (bz ? u[2] : 1.0 - u[2]);
        const double *e = &p->etab[4 * (((i0[0] + bx) * m + (i0[1] + by)) * m + (i0[2] + bz))];
        for (int q = 0; q < 4; q++)
            v[q] += w * e[q];
    }
    f[0] = sg[0] * v[0];
    f[1] = sg[1] * v[1];
    f[2] = sg[2] * v[2];
    *phi = v[3];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
