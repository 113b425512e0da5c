/*
 * Seeded synthetic silicon-pixel events.
 *
 * Produces the raw input of the reconstruction: packed digi words
 * (bits 0-7 row, 8-16 col, 17-24 ADC) with a 16-bit module id per digi,
 * plus per-module gain/pedestal tables.  It holds none of the
 * reconstruction arithmetic (no calibration, thresholds or clustering):
 * both the CPU oracle and the GPU path read what this file writes.
 *
 * Shapes follow the workload recipe of the pixel local-reconstruction
 * benchmark: random-walk charge blobs from a uniform seed, optional
 * 1 x L streaks along the column direction, uniform noise pixels,
 * "hot" modules filled with uniform pixels up to an occupancy, and
 * ADC = clamp(round(lognormal(mu, sigma)), 1, 255).  Duplicate
 * (module, row, col) positions are never emitted and the event is
 * shuffled so digis arrive unsorted across modules.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna) seeded through
 * splitmix64, Box-Muller normals, Knuth's product method for Poisson
 * draws (large means split into independent parts of at most 32).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} synth_rng;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(synth_rng *r, uint64_t seed)
{
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&seed);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(synth_rng *r)
{
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform double in [0, 1) */
static double rng_u01(synth_rng *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) (multiply-shift; the bias is below 2^-32) */
static uint32_t rng_below(synth_rng *r, uint32_t n)
{
    return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)n) >> 32);
}

static double rng_normal(synth_rng *r)
{
    double u1 = 1.0 - rng_u01(r); /* (0, 1] */
    double u2 = rng_u01(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static uint32_t poisson_small(synth_rng *r, double lam)
{
    const double L = exp(-lam);
    double p = 1.0;
    uint32_t k = 0;
    for (;;) {
        p *= rng_u01(r);
        if (p <= L) return k;
        ++k;
    }
}

static uint32_t rng_poisson(synth_rng *r, double lam)
{
    uint32_t k = 0;
    if (!(lam > 0.0)) return 0;
    while (lam > 32.0) {
        k += poisson_small(r, 32.0);
        lam -= 32.0;
    }
    return k + poisson_small(r, lam);
}

/* Per-event generation parameters (all per module unless stated). */
typedef struct synth_event_cfg {
    uint32_t n_modules, rows, cols;
    double lambda_clusters;  /* mean number of clusters in a module           */
    uint32_t n_inner;        /* modules 0..n_inner-1 draw at inner_factor x     */
    double inner_factor;
    uint32_t size_min, size_max; /* blob size in unique pixels, uniform        */
    uint32_t walk_cap;       /* maximum random-walk steps per blob            */
    double streak_frac;      /* probability that a cluster is a 1 x L streak  */
    uint32_t streak_len;
    double lambda_noise;     /* mean uniform noise pixels in a module          */
    double hot_frac;         /* fraction of modules that are "hot"             */
    double hot_occupancy;    /* pixel occupancy a hot module is filled to      */
    double adc_mu, adc_sigma;
} synth_event_cfg;

typedef struct {
    const synth_event_cfg *cfg;
    synth_rng *rng;
    uint8_t *occ;       /* occupancy bits of the current module */
    uint32_t *words;
    uint16_t *modules;
    uint64_t n, cap;
    uint32_t module;
    uint32_t in_module; /* digis emitted into the current module */
    int overflow;
} emitter;

static uint32_t draw_adc(emitter *e)
{
    double v = exp(e->cfg->adc_mu + e->cfg->adc_sigma * rng_normal(e->rng));
    double rd = floor(v + 0.5);
    if (rd < 1.0) rd = 1.0;
    if (rd > 255.0) rd = 255.0;
    return (uint32_t)rd;
}

static void emit(emitter *e, uint32_t row, uint32_t col)
{
    const uint32_t p = row * e->cfg->cols + col;
    if (e->occ[p >> 3] & (1u << (p & 7))) return; /* position already taken */
    if (e->n >= e->cap) {
        e->overflow = 1;
        return;
    }
    e->occ[p >> 3] |= (uint8_t)(1u << (p & 7));
    e->words[e->n] = row | (col << 8) | (draw_adc(e) << 17);
    e->modules[e->n] = (uint16_t)e->module;
    e->n++;
    e->in_module++;
}

static void emit_blob(emitter *e)
{
    const synth_event_cfg *c = e->cfg;
    static const int dr[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    static const int dc[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    uint32_t s = c->size_min + rng_below(e->rng, c->size_max - c->size_min + 1);
    uint32_t vis[512];
    uint32_t nvis = 0, steps = 0;
    int r = (int)rng_below(e->rng, c->rows);
    int col = (int)rng_below(e->rng, c->cols);
    if (s > 512) s = 512;
    vis[nvis++] = (uint32_t)r * c->cols + (uint32_t)col;
    while (nvis < s && steps < c->walk_cap) {
        uint32_t d = rng_below(e->rng, 8);
        r += dr[d];
        col += dc[d];
        if (r < 0) r = 0;
        if (r >= (int)c->rows) r = (int)c->rows - 1;
        if (col < 0) col = 0;
        if (col >= (int)c->cols) col = (int)c->cols - 1;
        ++steps;
        uint32_t p = (uint32_t)r * c->cols + (uint32_t)col;
        int seen = 0;
        for (uint32_t i = 0; i < nvis; ++i)
            if (vis[i] == p) {
                seen = 1;
                break;
            }
        if (!seen) vis[nvis++] = p;
    }
    for (uint32_t i = 0; i < nvis; ++i) emit(e, vis[i] / c->cols, vis[i] % c->cols);
}

static void emit_streak(emitter *e)
{
    const synth_event_cfg *c = e->cfg;
    uint32_t len = c->streak_len < c->cols ? c->streak_len : c->cols;
    uint32_t row = rng_below(e->rng, c->rows);
    uint32_t c0 = rng_below(e->rng, c->cols - len + 1);
    for (uint32_t i = 0; i < len; ++i) emit(e, row, c0 + i);
}

/*
 * Generate one event into words/modules (capacity cap).  Returns the number
 * of digis, or -1 if cap was too small.
 */
int64_t synth_event(const synth_event_cfg *cfg, uint64_t seed, uint32_t *words, uint16_t *modules,
                    uint64_t cap)
{
    synth_rng rng;
    rng_seed(&rng, seed);
    const uint32_t npix = cfg->rows * cfg->cols;
    const size_t occ_bytes = (npix + 7) / 8;
    uint8_t *occ = (uint8_t *)calloc(occ_bytes, 1);
    uint8_t *hot = (uint8_t *)calloc(cfg->n_modules ? cfg->n_modules : 1, 1);
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * (cfg->n_modules ? cfg->n_modules : 1));
    if (!occ || !hot || !perm) {
        free(occ);
        free(hot);
        free(perm);
        return -1;
    }
    /* choose the hot modules: a uniform subset of round(hot_frac * M) */
    uint32_t n_hot = (uint32_t)floor(cfg->hot_frac * cfg->n_modules + 0.5);
    for (uint32_t i = 0; i < cfg->n_modules; ++i) perm[i] = i;
    for (uint32_t i = 0; i < n_hot && i < cfg->n_modules; ++i) {
        uint32_t j = i + rng_below(&rng, cfg->n_modules - i);
        uint32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
        hot[perm[i]] = 1;
    }

    emitter e = {cfg, &rng, occ, words, modules, 0, cap, 0, 0, 0};
    for (uint32_t m = 0; m < cfg->n_modules; ++m) {
        e.module = m;
        e.in_module = 0;
        double lam = cfg->lambda_clusters * (m < cfg->n_inner ? cfg->inner_factor : 1.0);
        uint32_t k = rng_poisson(&rng, lam);
        for (uint32_t i = 0; i < k; ++i) {
            if (cfg->streak_frac > 0.0 && rng_u01(&rng) < cfg->streak_frac)
                emit_streak(&e);
            else
                emit_blob(&e);
        }
        uint32_t nn = rng_poisson(&rng, cfg->lambda_noise);
        for (uint32_t i = 0; i < nn; ++i) emit(&e, rng_below(&rng, cfg->rows), rng_below(&rng, cfg->cols));
        if (hot[m]) {
            uint32_t target = (uint32_t)floor(cfg->hot_occupancy * npix + 0.5);
            while (e.in_module < target && !e.overflow)
                emit(&e, rng_below(&rng, cfg->rows), rng_below(&rng, cfg->cols));
        }
        memset(occ, 0, occ_bytes);
        if (e.overflow) break;
    }
    free(occ);
    free(hot);
    free(perm);
    if (e.overflow) return -1;
    /* shuffle so that digis arrive unsorted across modules */
    for (uint64_t i = e.n; i > 1; --i) {
        uint64_t j = (uint64_t)(rng_u01(&rng) * (double)i);
        if (j >= i) j = i - 1;
        uint32_t tw = words[i - 1];
        words[i - 1] = words[j];
        words[j] = tw;
        uint16_t tm = modules[i - 1];
        modules[i - 1] = modules[j];
        modules[j] = tm;
    }
    return (int64_t)e.n;
}

/* Per-module calibration: gain uniform in [gain_lo, gain_hi], pedestal in [ped_lo, ped_hi]. */
void synth_calib(uint32_t n_modules, uint64_t seed, int32_t gain_lo, int32_t gain_hi, int32_t ped_lo,
                 int32_t ped_hi, int32_t *gain, int32_t *ped)
{
    synth_rng rng;
    rng_seed(&rng, seed);
    for (uint32_t m = 0; m < n_modules; ++m) {
        gain[m] = gain_lo + (int32_t)rng_below(&rng, (uint32_t)(gain_hi - gain_lo + 1));
        ped[m] = ped_lo + (int32_t)rng_below(&rng, (uint32_t)(ped_hi - ped_lo + 1));
    }
}

/* Uniform and lognormal helpers for per-event size draws (batched and serving workloads). */
void synth_uniform(uint64_t seed, uint64_t n, double lo, double hi, double *out)
{
    synth_rng rng;
    rng_seed(&rng, seed);
    for (uint64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * rng_u01(&rng);
}

void synth_lognormal(uint64_t seed, uint64_t n, double mu, double sigma, double *out)
{
    synth_rng rng;
    rng_seed(&rng, seed);
    for (uint64_t i = 0; i < n; ++i) out[i] = exp(mu + sigma * rng_normal(&rng));
}

/* Exponential inter-arrival gaps with the given rate (events per second). */
void synth_exponential(uint64_t seed, uint64_t n, double rate, double *out)
{
    synth_rng rng;
    rng_seed(&rng, seed);
    for (uint64_t i = 0; i < n; ++i) out[i] = -log(1.0 - rng_u01(&rng)) / rate;
}

/* splitmix64 mix of (base, index): independent per-event seeds. */
uint64_t synth_child_seed(uint64_t base, uint64_t index)
{
    uint64_t x = base ^ (0xA0761D6478BD642Full * (index + 1));
    splitmix64(&x);
    return splitmix64(&x);
}

/*
 * Synthetic barrel geometry for hits: module m sits on one of four layers
 * (radii 2.9, 6.8, 10.9, 16.0 cm), at azimuth phi and position z, facing
 * outwards.  Local coordinate u runs along the module's rows (global z),
 * v along its columns (the tangential direction).  origin[3m..] is the
 * module centre, rot[9m..] the row-major matrix R with global = origin +
 * R (u, v, 0).  Holds no reconstruction arithmetic.
 */
void synth_barrel_geometry(uint32_t n_modules, uint32_t rows, uint32_t cols, double pitch_row, double pitch_col,
                           float *origin, float *rot)
{
    static const double radius[4] = {2.9, 6.8, 10.9, 16.0};
    const double length = rows * pitch_row; /* along z */
    const uint32_t nz = 8;
    const uint32_t per_layer = (n_modules + 3) / 4;
    for (uint32_t m = 0; m < n_modules; ++m) {
        const uint32_t layer = m / per_layer, k = m % per_layer;
        const uint32_t nphi = (per_layer + nz - 1) / nz;
        const double phi = 6.283185307179586 * (double)(k % nphi) / (double)nphi;
        const double z = ((double)(k / nphi) - 0.5 * (double)(nz - 1)) * length;
        const double cp = cos(phi), sp = sin(phi);
        origin[3 * m + 0] = (float)(radius[layer] * cp);
        origin[3 * m + 1] = (float)(radius[layer] * sp);
        origin[3 * m + 2] = (float)z;
        float *R = rot + 9 * m;
        R[0] = 0.0f, R[1] = (float)-sp, R[2] = (float)cp;
        R[3] = 0.0f, R[4] = (float)cp, R[5] = (float)sp;
        R[6] = 1.0f, R[7] = 0.0f, R[8] = 0.0f;
        (void)cols;
    }
}
