/*
 * TEST INFRASTRUCTURE — the CPU oracle for silicon-pixel local reconstruction.
 *
 * A plain, slow, single-threaded restatement of what the offloaded
 * reconstruction computes, used only by the tests, the smoke check and the
 * benchmark's CPU-baseline leg to check and time the GPU library.  It shares
 * no code, header or table with the GPU path.
 *
 * The operation (the device workload that the paper's External Worker /
 * Product<T> / ScopedContext pattern of Sec. 2 and Sec. 4 carries; the
 * paper's Fig. 1 names it "raw -> clusters -> hits"), per event and per
 * module m, in this order:
 *   1. decode each digi word w: row = w & 0xFF, col = (w >> 8) & 0x1FF,
 *      adc = (w >> 17) & 0xFF; the digi is valid iff row < rows, col < cols,
 *      1 <= adc, (w >> 25) == 0 and module < n_modules, and no two digis share
 *      (module, row, col);
 *   2. calibrate: q = adc * gain[m] - pedestal[m] (int32); a pixel survives
 *      iff q >= pixel_thr;
 *   3. connected components of the surviving pixels of m under 8-adjacency
 *      (|drow| <= 1 and |dcol| <= 1, not both 0); no wrap at module edges,
 *      nothing joins across modules or events, dropped pixels do not bridge;
 *   4. per component: id = min over its pixels of row * cols + col;
 *      Q = sum q; npix; x = sum(q * row) / Q and y = sum(q * col) / Q with the
 *      sums exact in int64 and the division in double;
 *   5. keep the component iff Q >= cluster_thr;
 *   6. output kept clusters ordered by (module, id); label[i] of input digi i
 *      is the id of its kept cluster, -1 if it failed the pixel threshold, -2
 *      if its cluster failed the cluster threshold.
 * An event with an invalid digi reports ORACLE_EBADDIGI (checked first), one
 * with a duplicated position ORACLE_EDUP; such an event has no clusters and
 * all its labels are -1.  Thresholds and calibration must satisfy
 * pixel_thr >= 1, gain >= 0 and 255 * gain - pedestal <= INT32_MAX /
 * (rows * cols) (every charge sum then fits int32), else ORACLE_EINVAL.
 *
 * A second function, oracle_hits, takes the kept clusters one step further
 * along Fig. 1 (clusters -> hits): module placement turns each centroid into
 * a global position; its definition is written above the function.
 *
 * Step 3 is a textbook sequential union-find (path halving, link the root
 * of one tree under the other); the component id of step 4 is then the
 * smallest linear index found among the members, independent of how the
 * trees were linked.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    ORACLE_OK = 0,
    ORACLE_EINVAL = 3,
    ORACLE_EBADDIGI = 4,
    ORACLE_EDUP = 5,
    ORACLE_ECAPACITY = 6,
    ORACLE_ENOMEM = 7,
};

typedef struct oracle_geometry {
    uint32_t n_modules, rows, cols;
    int32_t pixel_thr, cluster_thr;
    const int32_t *gain;     /* [n_modules] */
    const int32_t *pedestal; /* [n_modules] */
} oracle_geometry;

typedef struct oracle_out {
    uint64_t capacity;   /* room in the cluster arrays */
    uint64_t n_clusters; /* written */
    uint32_t *module;
    int32_t *id, *charge, *npix;
    double *x, *y;
    int32_t *label; /* [n digis] */
} oracle_out;

static uint32_t uf_find(uint32_t *parent, uint32_t a)
{
    while (parent[a] != a) {
        parent[a] = parent[parent[a]];
        a = parent[a];
    }
    return a;
}

static void uf_union(uint32_t *parent, uint32_t a, uint32_t b)
{
    a = uf_find(parent, a);
    b = uf_find(parent, b);
    if (a != b) parent[a] = b;
}

typedef struct {
    int32_t id;
    int64_t Q;
    int32_t npix;
    int64_t sum_qr, sum_qc;
    uint32_t root;
} component;

static int cmp_component(const void *a, const void *b)
{
    int32_t x = ((const component *)a)->id, y = ((const component *)b)->id;
    return (x > y) - (x < y);
}

/*
 * Reconstruct one event of n digis.  Returns an ORACLE_* status; clusters and
 * labels go to *out.
 */
int oracle_event(const oracle_geometry *g, uint64_t n, const uint32_t *words, const uint16_t *modules,
                 oracle_out *out)
{
    const uint32_t M = g->n_modules, R = g->rows, C = g->cols;
    out->n_clusters = 0;
    for (uint64_t i = 0; i < n; ++i) out->label[i] = -1;
    if (g->pixel_thr < 1 || R == 0 || C == 0 || R > 256 || C > 512) return ORACLE_EINVAL;
    /* calibration domain: 0 <= gain and 255 * gain - pedestal <= INT32_MAX / (rows * cols),
       so that the charge of any cluster fits in int32 */
    for (uint32_t m = 0; m < M; ++m) {
        int64_t qmax = 255 * (int64_t)g->gain[m] - g->pedestal[m];
        if (g->gain[m] < 0 || qmax > (int64_t)INT32_MAX / ((int64_t)R * C)) return ORACLE_EINVAL;
    }

    /* step 1: decode and validate every digi */
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t w = words[i];
        uint32_t row = w & 0xFFu, col = (w >> 8) & 0x1FFu, adc = (w >> 17) & 0xFFu;
        if (row >= R || col >= C || adc < 1 || (w >> 25) != 0 || modules[i] >= M) return ORACLE_EBADDIGI;
    }

    /* bucket the digis by module (stable counting sort) */
    uint64_t *start = (uint64_t *)calloc((size_t)M + 1, sizeof(uint64_t));
    uint64_t *order = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    int64_t *grid = (int64_t *)malloc(sizeof(int64_t) * (size_t)R * C);
    uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    component *comp = (component *)malloc(sizeof(component) * (n ? n : 1));
    int32_t *comp_of_root = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
    if (!start || !order || !grid || !parent || !comp || !comp_of_root) {
        free(start), free(order), free(grid), free(parent), free(comp), free(comp_of_root);
        return ORACLE_ENOMEM;
    }
    for (uint64_t i = 0; i < n; ++i) start[modules[i] + 1]++;
    for (uint32_t m = 0; m < M; ++m) start[m + 1] += start[m];
    {
        uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)M + 1));
        memcpy(fill, start, sizeof(uint64_t) * ((size_t)M + 1));
        for (uint64_t i = 0; i < n; ++i) order[fill[modules[i]]++] = i;
        free(fill);
    }
    for (size_t p = 0; p < (size_t)R * C; ++p) grid[p] = -1;

    int status = ORACLE_OK;
    /* duplicates: any (module, row, col) seen twice */
    for (uint32_t m = 0; m < M && status == ORACLE_OK; ++m) {
        for (uint64_t k = start[m]; k < start[m + 1]; ++k) {
            uint32_t w = words[order[k]];
            size_t p = (size_t)(w & 0xFFu) * C + ((w >> 8) & 0x1FFu);
            if (grid[p] >= 0) status = ORACLE_EDUP;
            grid[p] = (int64_t)k;
        }
        for (uint64_t k = start[m]; k < start[m + 1]; ++k) {
            uint32_t w = words[order[k]];
            grid[(size_t)(w & 0xFFu) * C + ((w >> 8) & 0x1FFu)] = -1;
        }
    }

    for (uint32_t m = 0; m < M && status == ORACLE_OK; ++m) {
        const uint64_t b = start[m], e = start[m + 1];
        if (b == e) continue;
        /* step 2: calibrate; only surviving pixels enter the grid */
        for (uint64_t k = b; k < e; ++k) {
            uint32_t w = words[order[k]];
            int32_t adc = (int32_t)((w >> 17) & 0xFFu);
            int32_t q = adc * g->gain[m] - g->pedestal[m];
            parent[k - b] = (uint32_t)(k - b);
            if (q >= g->pixel_thr) grid[(size_t)(w & 0xFFu) * C + ((w >> 8) & 0x1FFu)] = (int64_t)k;
        }
        /* step 3: union each surviving pixel with its surviving 8-neighbours */
        for (uint64_t k = b; k < e; ++k) {
            uint32_t w = words[order[k]];
            int row = (int)(w & 0xFFu), col = (int)((w >> 8) & 0x1FFu);
            if (grid[(size_t)row * C + col] != (int64_t)k) continue; /* not a survivor */
            for (int dr = -1; dr <= 1; ++dr)
                for (int dc = -1; dc <= 1; ++dc) {
                    if (dr == 0 && dc == 0) continue;
                    int r2 = row + dr, c2 = col + dc;
                    if (r2 < 0 || r2 >= (int)R || c2 < 0 || c2 >= (int)C) continue;
                    int64_t nb = grid[(size_t)r2 * C + c2];
                    if (nb >= 0) uf_union(parent, (uint32_t)(k - b), (uint32_t)(nb - (int64_t)b));
                }
        }
        /* step 4: per-component id, charge, size and exact moment sums */
        uint64_t ncomp = 0;
        for (uint64_t k = b; k < e; ++k) comp_of_root[k - b] = -1;
        for (uint64_t k = b; k < e; ++k) {
            uint32_t w = words[order[k]];
            int64_t row = (int64_t)(w & 0xFFu), col = (int64_t)((w >> 8) & 0x1FFu);
            if (grid[(size_t)row * C + col] != (int64_t)k) continue;
            int64_t q = (int64_t)((w >> 17) & 0xFFu) * g->gain[m] - g->pedestal[m];
            uint32_t root = uf_find(parent, (uint32_t)(k - b));
            if (comp_of_root[root] < 0) {
                comp_of_root[root] = (int32_t)ncomp;
                comp[ncomp].id = INT32_MAX;
                comp[ncomp].Q = 0;
                comp[ncomp].npix = 0;
                comp[ncomp].sum_qr = comp[ncomp].sum_qc = 0;
                comp[ncomp].root = root;
                ncomp++;
            }
            component *c = &comp[comp_of_root[root]];
            int32_t lin = (int32_t)(row * C + col);
            if (lin < c->id) c->id = lin;
            c->Q += q;
            c->npix += 1;
            c->sum_qr += q * row;
            c->sum_qc += q * col;
        }
        /* steps 5-6: threshold, order by id, write clusters */
        qsort(comp, ncomp, sizeof(component), cmp_component);
        for (uint64_t j = 0; j < ncomp; ++j) comp_of_root[comp[j].root] = (int32_t)j;
        for (uint64_t j = 0; j < ncomp; ++j) {
            const component *c = &comp[j];
            if (c->Q < g->cluster_thr) continue;
            if (out->n_clusters >= out->capacity) {
                status = ORACLE_ECAPACITY;
                break;
            }
            uint64_t o = out->n_clusters++;
            out->module[o] = m;
            out->id[o] = c->id;
            out->charge[o] = (int32_t)c->Q;
            out->npix[o] = c->npix;
            out->x[o] = (double)c->sum_qr / (double)c->Q;
            out->y[o] = (double)c->sum_qc / (double)c->Q;
        }
        for (uint64_t k = b; k < e; ++k) {
            uint32_t w = words[order[k]];
            size_t p = (size_t)(w & 0xFFu) * C + ((w >> 8) & 0x1FFu);
            if (grid[p] != (int64_t)k) continue;
            const component *c = &comp[comp_of_root[uf_find(parent, (uint32_t)(k - b))]];
            out->label[order[k]] = c->Q >= g->cluster_thr ? c->id : -2;
        }
        for (uint64_t k = b; k < e; ++k) {
            uint32_t w = words[order[k]];
            grid[(size_t)(w & 0xFFu) * C + ((w >> 8) & 0x1FFu)] = -1;
        }
    }
    if (status != ORACLE_OK) {
        out->n_clusters = 0;
        for (uint64_t i = 0; i < n; ++i) out->label[i] = -1;
    }
    free(start), free(order), free(grid), free(parent), free(comp), free(comp_of_root);
    return status;
}

/*
 * A batch is the concatenation of independent events: event e owns digis
 * [offsets[e], offsets[e+1]).  Clusters are written event after event;
 * cluster_offsets[e] is the first cluster of event e (E+1 entries) and
 * status[e] the event's ORACLE_* status.  Returns the first non-OK status.
 */
int oracle_batch(const oracle_geometry *g, uint32_t n_events, const uint64_t *offsets, const uint32_t *words,
                 const uint16_t *modules, oracle_out *out, uint64_t *cluster_offsets, int32_t *status)
{
    int first = ORACLE_OK;
    uint64_t total = 0;
    for (uint32_t e = 0; e < n_events; ++e) {
        uint64_t a = offsets[e], b = offsets[e + 1];
        oracle_out o = *out;
        o.capacity = out->capacity - total;
        o.module += total, o.id += total, o.charge += total, o.npix += total, o.x += total, o.y += total;
        o.label = out->label + a;
        cluster_offsets[e] = total;
        int st = oracle_event(g, b - a, words + a, modules + a, &o);
        status[e] = st;
        if (st != ORACLE_OK && first == ORACLE_OK) first = st;
        total += o.n_clusters;
    }
    cluster_offsets[n_events] = total;
    out->n_clusters = total;
    return first;
}

/*
 * Hits: the clusters -> hits step of the paper's Fig. 1 (the GPU branch
 * produces hits from raw data directly).  A cluster of module m with
 * centroid (x, y) in pixel units (pixel (r, c) centred at (r, c)) has local
 * coordinates u = (x - (rows - 1) / 2) * pitch_row and
 * v = (y - (cols - 1) / 2) * pitch_col about the module centre, and global
 * position origin[m] + R[m] (u, v, 0), R[m] row-major.  Computed in double.
 */
void oracle_hits(uint32_t rows, uint32_t cols, double pitch_row, double pitch_col, const float *origin,
                 const float *rot, uint64_t n, const uint32_t *module, const double *x, const double *y,
                 double *gx, double *gy, double *gz)
{
    for (uint64_t i = 0; i < n; ++i) {
        const uint32_t m = module[i];
        const double u = (x[i] - 0.5 * (double)(rows - 1)) * pitch_row;
        const double v = (y[i] - 0.5 * (double)(cols - 1)) * pitch_col;
        const float *o = origin + 3 * (size_t)m;
        const float *R = rot + 9 * (size_t)m;
        gx[i] = (double)o[0] + (double)R[0] * u + (double)R[1] * v;
        gy[i] = (double)o[1] + (double)R[3] * u + (double)R[4] * v;
        gz[i] = (double)o[2] + (double)R[6] * u + (double)R[7] * v;
    }
}
