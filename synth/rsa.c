/*
 * Random sequential addition (RSA) of hard-core points into a slab of a
 * periodic orthorhombic box.  Workload construction only: it places atoms,
 * it computes nothing of the metadynamics method.
 *
 * Candidates are drawn from splitmix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), rounded to float32 (the
 * frame format) and accepted iff their minimum-image distance to every atom
 * already present is >= dmin.  Built with -ffp-contract=off and plain IEEE
 * double arithmetic so x86-64 and aarch64 produce identical frames.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t sm64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static double sm64_unit(uint64_t *state)
{
    return (double)(sm64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

static double min_image(double d, double L)
{
    if (d > 0.5 * L)
        d -= L;
    else if (d < -0.5 * L)
        d += L;
    return d;
}

typedef struct {
    int nc[3];
    double inv_h[3];
    int32_t *head; /* [ncells] */
    int32_t *next; /* [capacity] */
} grid_t;

static int cell_coord(double x, double inv_h, int nc)
{
    int c = (int)floor(x * inv_h);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

/* Offsets -1,0,1 collapse to the distinct cells when a dimension has fewer
 * than three cells, so no atom is visited twice. */
static int stencil(int nc, int *off)
{
    if (nc >= 3) { off[0] = -1; off[1] = 0; off[2] = 1; return 3; }
    if (nc == 2) { off[0] = 0; off[1] = 1; return 2; }
    off[0] = 0;
    return 1;
}

/*
 * Voxel bookkeeping: the sampling slab is cut into small voxels; a voxel is
 * "covered" once every point of it lies closer than dmin to one atom, so no
 * candidate inside it can ever be accepted.  Candidates are drawn uniformly
 * from the voxels not yet covered (uniform over a superset of the free
 * space), then tested exactly, which keeps the RSA distribution while
 * skipping most hopeless attempts near jamming.
 */
typedef struct {
    int nv[3];
    double e[3];
    double xlo;
    uint8_t *covered;
    int64_t *active;
    int64_t n_active;
    int64_t n_stale;
} voxels_t;

static void mark_atom(voxels_t *V, const double *box, double dmin, double px, double py, double pz)
{
    double d2 = dmin * dmin;
    double reach[3] = {dmin + V->e[0], dmin + V->e[1], dmin + V->e[2]};
    for (int kx = -1; kx <= 1; ++kx) {
        double ax = px + kx * box[0];
        int ix0 = (int)floor((ax - reach[0] - V->xlo) / V->e[0]);
        int ix1 = (int)floor((ax + reach[0] - V->xlo) / V->e[0]);
        if (ix1 < 0 || ix0 >= V->nv[0]) continue;
        if (ix0 < 0) ix0 = 0;
        if (ix1 >= V->nv[0]) ix1 = V->nv[0] - 1;
        int iy0 = (int)floor((py - reach[1]) / V->e[1]), iy1 = (int)floor((py + reach[1]) / V->e[1]);
        int iz0 = (int)floor((pz - reach[2]) / V->e[2]), iz1 = (int)floor((pz + reach[2]) / V->e[2]);
        for (int ix = ix0; ix <= ix1; ++ix) {
            double cx = fabs(V->xlo + (ix + 0.5) * V->e[0] - ax) + 0.5 * V->e[0];
            double fx = cx * cx;
            if (fx >= d2) continue;
            for (int iyr = iy0; iyr <= iy1; ++iyr) {
                double cy = fabs(min_image((iyr + 0.5) * V->e[1] - py, box[1])) + 0.5 * V->e[1];
                double fy = fx + cy * cy;
                if (fy >= d2) continue;
                int iy = ((iyr % V->nv[1]) + V->nv[1]) % V->nv[1];
                for (int izr = iz0; izr <= iz1; ++izr) {
                    double cz = fabs(min_image((izr + 0.5) * V->e[2] - pz, box[2])) + 0.5 * V->e[2];
                    if (fy + cz * cz >= d2) continue;
                    int iz = ((izr % V->nv[2]) + V->nv[2]) % V->nv[2];
                    int64_t id = ((int64_t)iz * V->nv[1] + iy) * V->nv[0] + ix;
                    if (!V->covered[id]) { V->covered[id] = 1; V->n_stale++; }
                }
            }
        }
    }
}

static void compact(voxels_t *V)
{
    int64_t k = 0;
    for (int64_t t = 0; t < V->n_active; ++t)
        if (!V->covered[V->active[t]]) V->active[k++] = V->active[t];
    V->n_active = k;
    V->n_stale = 0;
}

/*
 * exist_xyz: [n_exist][3] float32 atoms already placed (any position in box)
 * out_xyz:   [n_new][3]   float32 accepted points, x in [xlo, xhi)
 * Returns 0 on success, -1 on bad arguments, -2 when max_attempts is
 * exhausted or no free voxel is left (the caller fails loudly), -3 on
 * allocation failure.
 */
int synth_rsa_fill(int32_t n_exist, const float *exist_xyz, int32_t n_new,
                   float *out_xyz, const double *box, double xlo, double xhi,
                   double dmin, uint64_t seed, int64_t max_attempts,
                   int64_t *attempts_out)
{
    if (n_exist < 0 || n_new < 0 || dmin <= 0.0 || xhi <= xlo) return -1;
    grid_t g;
    int64_t ncells = 1;
    for (int d = 0; d < 3; ++d) {
        int nc = (int)floor(box[d] / dmin);
        if (nc < 1) nc = 1;
        g.nc[d] = nc;
        g.inv_h[d] = (double)nc / box[d];
        ncells *= nc;
    }
    voxels_t V;
    double span[3] = {xhi - xlo, box[1], box[2]};
    int64_t nvox = 1;
    for (int d = 0; d < 3; ++d) {
        V.nv[d] = (int)ceil(span[d] / (0.25 * dmin));
        V.e[d] = span[d] / V.nv[d];
        nvox *= V.nv[d];
    }
    V.xlo = xlo;
    int64_t cap = (int64_t)n_exist + n_new;
    g.head = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncells);
    g.next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    float *all = (float *)malloc(sizeof(float) * 3 * (size_t)(cap > 0 ? cap : 1));
    V.covered = (uint8_t *)calloc((size_t)nvox, 1);
    V.active = (int64_t *)malloc(sizeof(int64_t) * (size_t)nvox);
    if (!g.head || !g.next || !all || !V.covered || !V.active) {
        free(g.head); free(g.next); free(all); free(V.covered); free(V.active);
        return -3;
    }
    for (int64_t c = 0; c < ncells; ++c) g.head[c] = -1;
    memcpy(all, exist_xyz, sizeof(float) * 3 * (size_t)n_exist);
    int32_t n = 0;
    for (; n < n_exist; ++n) {
        int cx = cell_coord(all[3 * n + 0], g.inv_h[0], g.nc[0]);
        int cy = cell_coord(all[3 * n + 1], g.inv_h[1], g.nc[1]);
        int cz = cell_coord(all[3 * n + 2], g.inv_h[2], g.nc[2]);
        int64_t c = ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
        g.next[n] = g.head[c];
        g.head[c] = n;
        mark_atom(&V, box, dmin, all[3 * n + 0], all[3 * n + 1], all[3 * n + 2]);
    }
    V.n_active = 0;
    for (int64_t id = 0; id < nvox; ++id)
        if (!V.covered[id]) V.active[V.n_active++] = id;
    V.n_stale = 0;
    int ox[3], oy[3], oz[3];
    int sx = stencil(g.nc[0], ox), sy = stencil(g.nc[1], oy), sz = stencil(g.nc[2], oz);
    uint64_t st = seed;
    double d2min = dmin * dmin;
    int64_t attempts = 0;
    int32_t placed = 0;
    int rc = 0;
    while (placed < n_new) {
        if (V.n_stale * 2 > V.n_active) compact(&V);
        if (attempts >= max_attempts || V.n_active == 0) { rc = -2; break; }
        ++attempts;
        int64_t pick = (int64_t)(sm64_unit(&st) * (double)V.n_active);
        if (pick >= V.n_active) pick = V.n_active - 1;
        int64_t id = V.active[pick];
        double ux = sm64_unit(&st), uy = sm64_unit(&st), uz = sm64_unit(&st);
        if (V.covered[id]) continue;
        int64_t ix = id % V.nv[0], iy = (id / V.nv[0]) % V.nv[1], iz = id / ((int64_t)V.nv[0] * V.nv[1]);
        float px = (float)(xlo + (ix + ux) * V.e[0]);
        float py = (float)((iy + uy) * V.e[1]);
        float pz = (float)((iz + uz) * V.e[2]);
        if ((double)px < xlo || (double)px >= xhi || (double)py >= box[1] || (double)pz >= box[2]) continue;
        int cx = cell_coord(px, g.inv_h[0], g.nc[0]);
        int cy = cell_coord(py, g.inv_h[1], g.nc[1]);
        int cz = cell_coord(pz, g.inv_h[2], g.nc[2]);
        int ok = 1;
        for (int a = 0; a < sz && ok; ++a) {
            int zz = (cz + oz[a] + g.nc[2]) % g.nc[2];
            for (int b = 0; b < sy && ok; ++b) {
                int yy = (cy + oy[b] + g.nc[1]) % g.nc[1];
                for (int e = 0; e < sx && ok; ++e) {
                    int xx = (cx + ox[e] + g.nc[0]) % g.nc[0];
                    int64_t c = ((int64_t)zz * g.nc[1] + yy) * g.nc[0] + xx;
                    for (int32_t k = g.head[c]; k >= 0; k = g.next[k]) {
                        double dx = min_image((double)all[3 * k + 0] - (double)px, box[0]);
                        double dy = min_image((double)all[3 * k + 1] - (double)py, box[1]);
                        double dz = min_image((double)all[3 * k + 2] - (double)pz, box[2]);
                        double r2 = dx * dx + dy * dy;
                        r2 = r2 + dz * dz;
                        if (r2 < d2min) { ok = 0; break; }
                    }
                }
            }
        }
        if (!ok) continue;
        all[3 * n + 0] = px;
        all[3 * n + 1] = py;
        all[3 * n + 2] = pz;
        int64_t c = ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
        g.next[n] = g.head[c];
        g.head[c] = n;
        mark_atom(&V, box, dmin, px, py, pz);
        out_xyz[3 * placed + 0] = px;
        out_xyz[3 * placed + 1] = py;
        out_xyz[3 * placed + 2] = pz;
        ++n;
        ++placed;
    }
    *attempts_out = attempts;
    free(g.head); free(g.next); free(all); free(V.covered); free(V.active);
    return rc;
}
