/*
 * TEST INFRASTRUCTURE: a standalone driver for the CPU oracle, built with
 * AddressSanitizer and UndefinedBehaviorSanitizer by tests/test_oracle_sanitized.py.
 * Reads one batch (binary, little-endian) from argv[1], runs oracle_batch,
 * writes status, offsets and cluster arrays to argv[2].
 *
 * input:  u32 n_modules, rows, cols; i32 pixel_thr, cluster_thr; u32 E; u64 N;
 *         i32 gain[M]; i32 pedestal[M]; u64 offsets[E+1]; u32 words[N]; u16 modules[N]
 * output: i32 status; u64 C; u64 offsets[E+1]; i32 event_status[E]; u32 module[C];
 *         i32 id[C], charge[C], npix[C]; f64 x[C], y[C]; i32 label[N]
 */
#include <stdio.h>

#include "../oracle/hp_oracle.c"

static void *take(FILE *f, size_t bytes)
{
    void *p = malloc(bytes ? bytes : 1);
    if (!p || (bytes && fread(p, 1, bytes, f) != bytes)) exit(2);
    return p;
}

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    uint32_t hdr[3];
    int32_t thr[2];
    uint32_t E;
    uint64_t N;
    if (fread(hdr, 4, 3, f) != 3 || fread(thr, 4, 2, f) != 2 || fread(&E, 4, 1, f) != 1 || fread(&N, 8, 1, f) != 1)
        return 2;
    const uint32_t M = hdr[0];
    int32_t *gain = take(f, 4 * (size_t)M), *ped = take(f, 4 * (size_t)M);
    uint64_t *offs = take(f, 8 * ((size_t)E + 1));
    uint32_t *words = take(f, 4 * N);
    uint16_t *mods = take(f, 2 * N);
    fclose(f);
    oracle_geometry g = {M, hdr[1], hdr[2], thr[0], thr[1], gain, ped};
    const uint64_t cap = N ? N : 1;
    oracle_out o;
    o.capacity = cap;
    o.n_clusters = 0;
    o.module = malloc(4 * cap);
    o.id = malloc(4 * cap);
    o.charge = malloc(4 * cap);
    o.npix = malloc(4 * cap);
    o.x = malloc(8 * cap);
    o.y = malloc(8 * cap);
    o.label = malloc(4 * cap);
    uint64_t *coff = calloc((size_t)E + 1, 8);
    int32_t *est = calloc(E ? E : 1, 4);
    const int32_t st = oracle_batch(&g, E, offs, words, mods, &o, coff, est);
    FILE *w = fopen(argv[2], "wb");
    if (!w) return 2;
    const uint64_t C = o.n_clusters;
    fwrite(&st, 4, 1, w);
    fwrite(&C, 8, 1, w);
    fwrite(coff, 8, (size_t)E + 1, w);
    fwrite(est, 4, E, w);
    fwrite(o.module, 4, C, w);
    fwrite(o.id, 4, C, w);
    fwrite(o.charge, 4, C, w);
    fwrite(o.npix, 4, C, w);
    fwrite(o.x, 8, C, w);
    fwrite(o.y, 8, C, w);
    fwrite(o.label, 4, N, w);
    fclose(w);
    free(gain);
    free(ped);
    free(offs);
    free(words);
    free(mods);
    free(o.module);
    free(o.id);
    free(o.charge);
    free(o.npix);
    free(o.x);
    free(o.y);
    free(o.label);
    free(coff);
    free(est);
    return 0;
}
