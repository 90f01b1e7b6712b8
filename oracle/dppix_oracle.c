/*
 * dppix_oracle.c -- CPU oracle for region-adaptive differentially private pixelization.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the CUDA path is
 * checked against.  Only the test suite, the package smoke check and the CPU-baseline leg of the benchmark
 * may load it; the product library never links, calls or falls back to it.  It shares no code, header,
 * table or constant with the CUDA sources.
 *
 * Everything is computed in double precision with exact 64-bit integer pixel sums, cell by cell, in the
 * order the paper states the method:
 *   - pixelization: b x b cell means broadcast over the cell (Sec. IV-A, Eq. 1-4);
 *   - Laplace mechanism: sigma = sensitivity / eps, eta ~ Laplace(0, sigma) (Sec. IV-B, Eq. 7-9);
 *   - sensitivity of the pixelization 255*m/b^2 -- here R*m/b^2 for a value range R (Sec. IV-D, Eq. 11);
 *   - noisy mean clipped to [0, R] (Sec. IV-D; Alg. 1 and Alg. 2);
 *   - mirror padding to whole grids, mean, noise, clip, repeat, crop (Alg. 2);
 *   - mask mean per grid, simple (> 1/2) / complex (<= 1/2) split, per-region grid and noise (Alg. 3,
 *     Sec. VI-A..D, Eq. 16-17), generalised to K regions on tiles of side T = lcm{b_r};
 *   - compact record of noisy statistics and reconstruction by broadcast (Table III, Table IV, Sec. VI-F).
 *
 * Readings of points the paper leaves open (channels, tie rule, sampler, keying, record layout, variance
 * classes, soft layer) are the ones listed for this build; each function names the reading it follows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------------ */
/* Error codes (the oracle's own; negative = error)                                                  */
/* ------------------------------------------------------------------------------------------------ */
enum {
    ORA_OK = 0,
    ORA_E_INVALID = -1,
    ORA_E_PAD = -2,
    ORA_E_SMALL = -3,
    ORA_E_RECORD = -4,
    ORA_E_NOMEM = -5
};

/* ------------------------------------------------------------------------------------------------ */
/* Philox4xW-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).                         */
/* One macro defines both word widths so that the 64-bit instance (checked against numpy's Philox)   */
/* pins the round and key-schedule structure shared with the 32-bit instance used for the noise.     */
/* ------------------------------------------------------------------------------------------------ */
static void mulhilo_32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

static void mulhilo_64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

#define ORA_DEFINE_PHILOX4(WBITS, WT, MUL0, MUL1, BUMP0, BUMP1)                                   \
    void ora_philox4x##WBITS##_10(const WT ctr[4], const WT key[2], WT out[4])                     \
    {                                                                                              \
        WT x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];                                     \
        WT k0 = key[0], k1 = key[1];                                                               \
        for (int round = 0; round < 10; ++round) {                                                 \
            if (round > 0) { /* key schedule: Weyl increments between rounds */                   \
                k0 = (WT)(k0 + (BUMP0));                                                           \
                k1 = (WT)(k1 + (BUMP1));                                                           \
            }                                                                                      \
            WT hi0, lo0, hi1, lo1;                                                                 \
            mulhilo_##WBITS((MUL0), x0, &hi0, &lo0);                                               \
            mulhilo_##WBITS((MUL1), x2, &hi1, &lo1);                                               \
            WT y0 = hi1 ^ x1 ^ k0;                                                                 \
            WT y1 = lo1;                                                                           \
            WT y2 = hi0 ^ x3 ^ k1;                                                                 \
            WT y3 = lo0;                                                                           \
            x0 = y0; x1 = y1; x2 = y2; x3 = y3;                                                    \
        }                                                                                          \
        out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;                                        \
    }

/* multipliers and Weyl constants as published for Philox4x32 and Philox4x64 */
ORA_DEFINE_PHILOX4(32, uint32_t, 0xD2511F53u, 0xCD9E8D57u, 0x9E3779B9u, 0xBB67AE85u)
ORA_DEFINE_PHILOX4(64, uint64_t, 0xD2E7470EE14C6C93ull, 0xCA5A826395121157ull,
                   0x9E3779B97F4A7C15ull, 0xBB67AE8584CAA73Bull)

/*
 * Laplace(0, sigma) draw from one uniform 32-bit word x by the inverse CDF (Eq. 9; sampler reading):
 * u = (x + 1/2) / 2^32.  For u < 1/2 the inverse CDF is sigma*ln(2u); for u >= 1/2 it is -sigma*ln(2(1-u)).
 * Both arguments are t = (k + 1/2) / 2^31 with k = x or k = 2^32-1-x, which is exact in double.
 */
double ora_laplace_from_word(uint32_t x, double sigma)
{
    if (x < 0x80000000u) {
        double t = ((double)x + 0.5) / 2147483648.0;
        return sigma * log(t);
    } else {
        uint32_t k = 0xFFFFFFFFu - x;
        double t = ((double)k + 0.5) / 2147483648.0;
        return -sigma * log(t);
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Problem description and derived geometry                                                          */
/* ------------------------------------------------------------------------------------------------ */
#define ORA_MAXK 8

typedef struct {
    int32_t M, N, C;          /* frame height, width, channels (interleaved u8 samples) */
    int32_t K;                /* number of regions */
    int64_t pitch;            /* bytes between frame rows */
    int32_t b[ORA_MAXK];      /* grid side of region r */
    double eps[ORA_MAXK];     /* privacy budget of region r */
    double R;                 /* value range (255 for u8) */
    double m;                 /* max number of differing samples between neighbouring images */
    int32_t pad_mode;         /* 0 = reflect (edge not repeated), 1 = symmetric (edge repeated) */
    int32_t source;           /* 0 tile labels, 1 simple-mask u8, 2 alpha matte f32, 3 variance quantiles */
    float matte_thr;          /* matte pixel is complex iff alpha >= matte_thr */
    int32_t dtype;            /* record payload: 0 f32 means, 1 u8 means, 2 u32 raw sums */
    int32_t noise_free;       /* 1: eta = 0 (the eps -> infinity limit) */
    uint32_t stream_id;
    uint64_t seed;
    uint64_t frame_idx;
} ora_desc;

typedef struct {
    int32_t T, GR, GC, PR, PC;
    int32_t cells_side[ORA_MAXK];   /* T / b_r */
    double sigma[ORA_MAXK];
    uint64_t header_bytes, rowidx_bytes, map_offset, payload_offset, capacity;
} ora_geom;

static int64_t gcd64(int64_t a, int64_t b)
{
    while (b) { int64_t t = a % b; a = b; b = t; }
    return a;
}

/* Record header byte offsets (the documented record format, written out here independently). */
enum {
    H_MAGIC = 0, H_VERSION = 4, H_HBYTES = 8, H_FLAGS = 12, H_M = 16, H_N = 20, H_C = 24, H_T = 28,
    H_K = 32, H_GR = 36, H_GC = 40, H_PAD = 44, H_DTYPE = 48, H_SOURCE = 52, H_STREAM = 56,
    H_SEED = 64, H_FRAME = 72, H_R = 80, H_MM = 88, H_TOTAL = 96, H_MAPOFF = 104, H_B = 112,
    H_EPS = 144, H_SIGMA = 208, H_COUNT = 272, H_ROFF = 304, H_ROWOFF = 368, H_PAYOFF = 376,
    H_SIZE = 512
};

static uint64_t align16(uint64_t x) { return (x + 15u) & ~(uint64_t)15u; }

static int dtype_bytes(int dtype) { return dtype == 1 ? 1 : 4; }

/* Sec. V-B: Alg. 2 steps 1-3 and Alg. 3 steps 1-2, with T = lcm{b_r} as the tile (the paper's b when one
 * region's grid divides the other's, Eq. 16). sigma_r = R*m/(b_r^2 eps_r) (Eq. 11 with Eq. 8). */
int ora_geometry(const ora_desc *d, ora_geom *g)
{
    if (!d || !g) return ORA_E_INVALID;
    memset(g, 0, sizeof(*g));
    if (d->M < 1 || d->N < 1 || d->C < 1 || d->C > 4 || d->K < 1 || d->K > ORA_MAXK) return ORA_E_INVALID;
    if (d->pitch < (int64_t)d->N * d->C) return ORA_E_INVALID;
    if (!(d->R > 0) || !(d->m > 0)) return ORA_E_INVALID;
    if (d->pad_mode < 0 || d->pad_mode > 2) return ORA_E_INVALID;
    /* pad mode 2 (no padding, valid samples only) ranks no tile variances: tiles would hold unequal counts */
    if (d->pad_mode == 2 && d->source == 3) return ORA_E_INVALID;
    if (d->dtype < 0 || d->dtype > 2) return ORA_E_INVALID;
    if (d->source < 0 || d->source > 3) return ORA_E_INVALID;
    if ((d->source == 1 || d->source == 2) && d->K != 2) return ORA_E_INVALID;
    int64_t T = 1;
    for (int r = 0; r < d->K; ++r) {
        if (d->b[r] < 1) return ORA_E_INVALID;
        if (!d->noise_free && !(d->eps[r] > 0)) return ORA_E_INVALID;
        T = T / gcd64(T, d->b[r]) * d->b[r];
        if (T > 4096) return ORA_E_INVALID;
    }
    g->T = (int32_t)T;
    g->GR = (int32_t)((d->M + T - 1) / T);
    g->GC = (int32_t)((d->N + T - 1) / T);
    g->PR = (int32_t)(g->GR * T - d->M);
    g->PC = (int32_t)(g->GC * T - d->N);
    /* mirror padding must stay inside the image: reflect needs P <= n-1, symmetric P <= n (mode 2 pads nothing) */
    int64_t lim_r = d->pad_mode == 0 ? d->M - 1 : d->M;
    int64_t lim_c = d->pad_mode == 0 ? d->N - 1 : d->N;
    if (d->pad_mode != 2 && (g->PR > lim_r || g->PC > lim_c)) return ORA_E_PAD;
    for (int r = 0; r < d->K; ++r) {
        g->cells_side[r] = (int32_t)(T / d->b[r]);
        g->sigma[r] = d->R * d->m / ((double)d->b[r] * (double)d->b[r] * d->eps[r]);
    }
    uint64_t ntiles = (uint64_t)g->GR * (uint64_t)g->GC;
    g->header_bytes = H_SIZE;
    g->rowidx_bytes = align16((uint64_t)g->GR * (uint64_t)d->K * 4u);
    g->map_offset = g->header_bytes + g->rowidx_bytes;
    g->payload_offset = g->map_offset + align16(ntiles);
    uint64_t maxcells = 0;
    for (int r = 0; r < d->K; ++r) {
        uint64_t c = (uint64_t)g->cells_side[r] * (uint64_t)g->cells_side[r];
        if (c > maxcells) maxcells = c;
    }
    g->capacity = g->payload_offset + align16(ntiles * maxcells * (uint64_t)d->C * dtype_bytes(d->dtype)) +
                  16u * (uint64_t)d->K;
    return ORA_OK;
}

/* Mirror padding by index (Alg. 2 step 4, Alg. 3 step 3): padded index p >= n maps back into [0, n).
 * reflect: the edge sample is not repeated (p -> 2(n-1) - p); symmetric: it is (p -> 2n - 1 - p). */
int64_t ora_reflect(int64_t p, int64_t n, int pad_mode)
{
    if (p < n) return p;
    return pad_mode == 0 ? 2 * (n - 1) - p : 2 * n - 1 - p;
}

static int sample_u8(const ora_desc *d, const uint8_t *img, int64_t y, int64_t x, int ch)
{
    int64_t sy = ora_reflect(y, d->M, d->pad_mode);
    int64_t sx = ora_reflect(x, d->N, d->pad_mode);
    return img[sy * d->pitch + sx * d->C + ch];
}

/* ------------------------------------------------------------------------------------------------ */
/* Tile classification (Alg. 3 steps 5-6 and the region sources of this build)                       */
/* ------------------------------------------------------------------------------------------------ */
typedef struct { uint64_t key_hi, key_lo; int64_t idx; } ora_rank_item;

static int cmp_rank_item(const void *a, const void *b)
{
    const ora_rank_item *p = (const ora_rank_item *)a, *q = (const ora_rank_item *)b;
    if (p->key_hi != q->key_hi) return p->key_hi < q->key_hi ? -1 : 1;
    if (p->key_lo != q->key_lo) return p->key_lo < q->key_lo ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

/*
 * Writes the G_R x G_C region map (row-major, one u8 region id per T x T tile).
 *  source 0: tile labels given by the caller (src = u8 G_R x G_C, values < K), copied.
 *  source 1: simple-region mask M (Alg. 3 input; nonzero = simple), padded like the image.  The mask mean
 *            of the tile is > 1/2 (simple, region 0) or <= 1/2 (complex, region 1) -- Alg. 3 step 6, taken
 *            on integer counts: simple iff 2 * (#simple samples) > T^2, so a tie goes to complex.
 *  source 2: alpha matte (f32); a pixel is complex iff alpha >= matte_thr, then as source 1.
 *  source 3: local-variance quantile classes: per tile S = sum x, Q = sum x^2 over the C*T^2 padded samples,
 *            key = n*Q - S^2 (n^2 times the variance, exact), tiles ranked ascending by (key, tile index),
 *            class q = floor(K * rank / #tiles), region q (lowest variance = region 0).
 * src_pitch is in bytes (rows of the mask / matte); ignored for source 0 and 3.
 */
int ora_classify(const ora_desc *d, const uint8_t *img, const void *src, int64_t src_pitch, uint8_t *map)
{
    ora_geom g;
    int rc = ora_geometry(d, &g);
    if (rc) return rc;
    const int64_t T = g.T, GR = g.GR, GC = g.GC, ntiles = GR * GC;
    if (d->source == 0) {
        const uint8_t *lab = (const uint8_t *)src;
        for (int64_t i = 0; i < ntiles; ++i) {
            if (lab[i] >= d->K) return ORA_E_INVALID;
            map[i] = lab[i];
        }
        return ORA_OK;
    }
    if (d->source == 1 || d->source == 2) {
        for (int64_t ty = 0; ty < GR; ++ty)
            for (int64_t tx = 0; tx < GC; ++tx) {
                int64_t simple = 0;
                /* mode 2: only the tile's samples inside the frame count, and the mean is over them */
                const int64_t y1 = d->pad_mode == 2 && (ty + 1) * T > d->M ? d->M : (ty + 1) * T;
                const int64_t x1 = d->pad_mode == 2 && (tx + 1) * T > d->N ? d->N : (tx + 1) * T;
                const int64_t nvalid = (y1 - ty * T) * (x1 - tx * T);
                for (int64_t y = ty * T; y < y1; ++y)
                    for (int64_t x = tx * T; x < x1; ++x) {
                        int64_t sy = ora_reflect(y, d->M, d->pad_mode);
                        int64_t sx = ora_reflect(x, d->N, d->pad_mode);
                        int is_simple;
                        if (d->source == 1) {
                            is_simple = ((const uint8_t *)src)[sy * src_pitch + sx] != 0;
                        } else {
                            const float *row = (const float *)((const uint8_t *)src + sy * src_pitch);
                            is_simple = !(row[sx] >= d->matte_thr);
                        }
                        simple += is_simple;
                    }
                map[ty * GC + tx] = (2 * simple > nvalid) ? 0 : 1;
            }
        return ORA_OK;
    }
    /* source 3 */
    ora_rank_item *items = (ora_rank_item *)malloc(sizeof(ora_rank_item) * (size_t)ntiles);
    if (!items) return ORA_E_NOMEM;
    const unsigned __int128 n = (unsigned __int128)(d->C * T * T);
    for (int64_t ty = 0; ty < GR; ++ty)
        for (int64_t tx = 0; tx < GC; ++tx) {
            uint64_t S = 0, Q = 0;
            for (int64_t y = ty * T; y < (ty + 1) * T; ++y)
                for (int64_t x = tx * T; x < (tx + 1) * T; ++x)
                    for (int ch = 0; ch < d->C; ++ch) {
                        uint64_t v = (uint64_t)sample_u8(d, img, y, x, ch);
                        S += v;
                        Q += v * v;
                    }
            unsigned __int128 key = n * (unsigned __int128)Q - (unsigned __int128)S * (unsigned __int128)S;
            ora_rank_item *it = &items[ty * GC + tx];
            it->key_hi = (uint64_t)(key >> 64);
            it->key_lo = (uint64_t)key;
            it->idx = ty * GC + tx;
        }
    qsort(items, (size_t)ntiles, sizeof(ora_rank_item), cmp_rank_item);
    for (int64_t rank = 0; rank < ntiles; ++rank)
        map[items[rank].idx] = (uint8_t)((int64_t)d->K * rank / ntiles);
    free(items);
    return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Little-endian scalar writers / readers for the record                                             */
/* ------------------------------------------------------------------------------------------------ */
static void put_u32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_u64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_f64(uint8_t *p, double v) { uint64_t u; memcpy(&u, &v, 8); put_u64(p, u); }
static void put_f32(uint8_t *p, float v) { uint32_t u; memcpy(&u, &v, 4); put_u32(p, u); }
static uint32_t get_u32(const uint8_t *p)
{
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
static uint64_t get_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}
static float get_f32(const uint8_t *p) { uint32_t u = get_u32(p); float f; memcpy(&f, &u, 4); return f; }

/* ------------------------------------------------------------------------------------------------ */
/* Release: classify, then per region, per tile, per cell, per channel: exact sum, mean, noise, clip  */
/* ------------------------------------------------------------------------------------------------ */

/* Exact integer sum of one b x b cell of channel ch over the mirror-padded image (Eq. 2, Alg. 2 step 6). */
static int64_t cell_sum(const ora_desc *d, const uint8_t *img, int64_t y0, int64_t x0, int64_t b, int ch)
{
    int64_t s = 0;
    for (int64_t y = y0; y < y0 + b; ++y)
        for (int64_t x = x0; x < x0 + b; ++x) s += sample_u8(d, img, y, x, ch);
    return s;
}

/*
 * Full release of one frame into a record (Alg. 3 generalised to K regions; record per Table IV).
 * Record order: region-major (the paper stores mu'_G, then mu'_Gs), then tiles of that region in row-major
 * tile order, then cells row-major inside the tile, then the C channels.
 * Noise key (sampler reading): Philox4x32-10 with key (seed mod 2^32, seed >> 32) and counter
 * (cell index in the padded b_r-grid of the frame, r | stream << 8, frame mod 2^32, frame >> 32);
 * output word ch is the draw for channel ch.
 * means_out / sums_out (optional) receive, in record order, the fp64 clipped noisy means and exact sums.
 */
int ora_release(const ora_desc *d, const uint8_t *img, const void *src, int64_t src_pitch,
                uint8_t *rec, uint64_t cap, double *means_out, int64_t *sums_out, double *eta_out)
{
    ora_geom g;
    int rc = ora_geometry(d, &g);
    if (rc) return rc;
    if (d->stream_id >= (1u << 24)) return ORA_E_INVALID;
    const int64_t T = g.T, GR = g.GR, GC = g.GC, ntiles = GR * GC, C = d->C;
    if (cap < g.capacity) return ORA_E_SMALL;
    uint8_t *map = (uint8_t *)malloc((size_t)ntiles);
    if (!map) return ORA_E_NOMEM;
    rc = ora_classify(d, img, src, src_pitch, map);
    if (rc) { free(map); return rc; }

    memset(rec, 0, (size_t)g.payload_offset);
    uint64_t count[ORA_MAXK] = {0};
    for (int64_t i = 0; i < ntiles; ++i) count[map[i]]++;
    uint64_t roff[ORA_MAXK];
    uint64_t off = g.payload_offset;
    const int es = dtype_bytes(d->dtype);
    for (int r = 0; r < d->K; ++r) {
        roff[r] = off;
        uint64_t cells = (uint64_t)g.cells_side[r] * (uint64_t)g.cells_side[r];
        off = align16(off + count[r] * cells * (uint64_t)C * (uint64_t)es);
    }
    const uint64_t total = off;

    /* header */
    memcpy(rec + H_MAGIC, "DPPX", 4);
    put_u32(rec + H_VERSION, 1);
    put_u32(rec + H_HBYTES, H_SIZE);
    put_u32(rec + H_FLAGS, d->noise_free ? 1u : 0u);
    put_u32(rec + H_M, (uint32_t)d->M);
    put_u32(rec + H_N, (uint32_t)d->N);
    put_u32(rec + H_C, (uint32_t)d->C);
    put_u32(rec + H_T, (uint32_t)T);
    put_u32(rec + H_K, (uint32_t)d->K);
    put_u32(rec + H_GR, (uint32_t)GR);
    put_u32(rec + H_GC, (uint32_t)GC);
    put_u32(rec + H_PAD, (uint32_t)d->pad_mode);
    put_u32(rec + H_DTYPE, (uint32_t)d->dtype);
    put_u32(rec + H_SOURCE, (uint32_t)d->source);
    put_u32(rec + H_STREAM, d->stream_id);
    put_u64(rec + H_SEED, d->seed);
    put_u64(rec + H_FRAME, d->frame_idx);
    put_f64(rec + H_R, d->R);
    put_f64(rec + H_MM, d->m);
    put_u64(rec + H_TOTAL, total);
    put_u64(rec + H_MAPOFF, g.map_offset);
    for (int r = 0; r < d->K; ++r) {
        put_u32(rec + H_B + 4 * r, (uint32_t)d->b[r]);
        put_f64(rec + H_EPS + 8 * r, d->eps[r]);
        put_f64(rec + H_SIGMA + 8 * r, g.sigma[r]);
        put_u32(rec + H_COUNT + 4 * r, (uint32_t)count[r]);
        put_u64(rec + H_ROFF + 8 * r, roff[r]);
    }
    put_u64(rec + H_ROWOFF, g.header_bytes);
    put_u64(rec + H_PAYOFF, g.payload_offset);
    /* tile-row index: number of region-r tiles in tile rows above ty */
    {
        uint64_t run[ORA_MAXK] = {0};
        for (int64_t ty = 0; ty < GR; ++ty) {
            for (int r = 0; r < d->K; ++r) put_u32(rec + g.header_bytes + 4 * (ty * d->K + r), (uint32_t)run[r]);
            for (int64_t tx = 0; tx < GC; ++tx) run[map[ty * GC + tx]]++;
        }
    }
    memcpy(rec + g.map_offset, map, (size_t)ntiles);
    memset(rec + g.payload_offset, 0, (size_t)(total - g.payload_offset));

    /* payload, region-major */
    uint64_t k = 0; /* running element index in record order (for the optional fp64 outputs) */
    for (int r = 0; r < d->K; ++r) {
        const int64_t b = d->b[r], cs = g.cells_side[r];
        const int64_t grid_w = GC * cs; /* cells per row of the padded b_r-grid */
        const double inv_b2 = 1.0 / ((double)b * (double)b);
        uint64_t e = 0; /* element index within region r */
        for (int64_t ty = 0; ty < GR; ++ty)
            for (int64_t tx = 0; tx < GC; ++tx) {
                if (map[ty * GC + tx] != r) continue;
                for (int64_t cy = 0; cy < cs; ++cy)
                    for (int64_t cx = 0; cx < cs; ++cx) {
                        const int64_t gy = ty * cs + cy, gx = tx * cs + cx;
                        uint32_t ctr[4] = {(uint32_t)(gy * grid_w + gx), (uint32_t)r | (d->stream_id << 8),
                                           (uint32_t)d->frame_idx, (uint32_t)(d->frame_idx >> 32)};
                        uint32_t key[2] = {(uint32_t)d->seed, (uint32_t)(d->seed >> 32)};
                        uint32_t words[4];
                        ora_philox4x32_10(ctr, key, words);
                        /* pad mode 2 (Alg. 1 semantics): an edge cell holds h x w samples inside the frame; its mean
                         * is over them and its noise scale R m / (h w eps_r) (Eq. 11 with h w in place of b^2); a cell
                         * wholly outside the frame holds no sample and stores 0 */
                        int64_t h = b, w = b;
                        if (d->pad_mode == 2) {
                            h = d->M - gy * b;
                            w = d->N - gx * b;
                            h = h < 0 ? 0 : (h > b ? b : h);
                            w = w < 0 ? 0 : (w > b ? b : w);
                        }
                        const int64_t n = h * w;
                        const double sigma_c = d->R * d->m / ((double)n * d->eps[r]);
                        for (int ch = 0; ch < C; ++ch, ++e, ++k) {
                            int64_t S;
                            double mu, eta, v;
                            if (d->pad_mode != 2) {
                                S = cell_sum(d, img, gy * b, gx * b, b, ch);
                                mu = (double)S * inv_b2;
                                eta = d->noise_free ? 0.0 : ora_laplace_from_word(words[ch], g.sigma[r]);
                            } else {
                                S = 0;
                                for (int64_t y = gy * b; y < gy * b + h; ++y)
                                    for (int64_t x = gx * b; x < gx * b + w; ++x) S += img[y * d->pitch + x * C + ch];
                                mu = n ? (double)S / (double)n : 0.0;
                                eta = (d->noise_free || n == 0) ? 0.0 : ora_laplace_from_word(words[ch], sigma_c);
                            }
                            v = mu + eta;
                            if (v < 0.0) v = 0.0;
                            if (v > d->R) v = d->R;
                            uint8_t *dst = rec + roff[r] + e * (uint64_t)es;
                            if (d->dtype == 0) put_f32(dst, (float)v);
                            else if (d->dtype == 1) *dst = (uint8_t)rintf((float)v);
                            else put_u32(dst, (uint32_t)S);
                            if (means_out) means_out[k] = v;
                            if (sums_out) sums_out[k] = S;
                            if (eta_out) eta_out[k] = eta;
                        }
                    }
            }
    }
    free(map);
    return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Reconstruction from a record alone (Sec. VI-F: metadata suffice; Alg. 2 steps 10-11).              */
/* ------------------------------------------------------------------------------------------------ */

/* Reads the geometry out of a record header; checks the fields the reconstruction relies on. */
int ora_record_info(const uint8_t *rec, uint64_t len, int32_t out[16])
{
    if (len < H_SIZE || memcmp(rec, "DPPX", 4) != 0 || get_u32(rec + H_VERSION) != 1) return ORA_E_RECORD;
    out[0] = (int32_t)get_u32(rec + H_M);
    out[1] = (int32_t)get_u32(rec + H_N);
    out[2] = (int32_t)get_u32(rec + H_C);
    out[3] = (int32_t)get_u32(rec + H_T);
    out[4] = (int32_t)get_u32(rec + H_K);
    out[5] = (int32_t)get_u32(rec + H_GR);
    out[6] = (int32_t)get_u32(rec + H_GC);
    out[7] = (int32_t)get_u32(rec + H_DTYPE);
    uint64_t total = get_u64(rec + H_TOTAL);
    if (total > len) return ORA_E_RECORD;
    out[8] = (int32_t)(total & 0x7fffffff);
    return ORA_OK;
}

/*
 * out_type 0: u8 image M x N x C (round half to even of the stored value), out_pitch bytes per row.
 * out_type 1: f32 image, out_pitch bytes per row.  out_type 2: f64 image.
 * A record of exact sums (dtype 2) reconstructs to the noise-free block means.
 * The tile-row index stored in the record is recomputed from the map and must agree.
 */
int ora_reconstruct(const uint8_t *rec, uint64_t len, int out_type, void *out, int64_t out_pitch)
{
    int32_t info[16];
    int rc = ora_record_info(rec, len, info);
    if (rc) return rc;
    const int64_t M = info[0], N = info[1], C = info[2], T = info[3], K = info[4], GR = info[5], GC = info[6];
    const int dtype = info[7];
    if (C < 1 || C > 4 || K < 1 || K > ORA_MAXK || T < 1 || GR != (M + T - 1) / T || GC != (N + T - 1) / T)
        return ORA_E_RECORD;
    const uint64_t map_off = get_u64(rec + H_MAPOFF), row_off = get_u64(rec + H_ROWOFF);
    const uint8_t *map = rec + map_off;
    int64_t b[ORA_MAXK];
    uint64_t roff[ORA_MAXK];
    for (int r = 0; r < K; ++r) {
        b[r] = get_u32(rec + H_B + 4 * r);
        roff[r] = get_u64(rec + H_ROFF + 8 * r);
        if (b[r] < 1 || T % b[r] != 0) return ORA_E_RECORD;
    }
    /* index of each tile within its region, by a plain scan of the map in row-major order */
    int64_t ntiles = GR * GC;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)ntiles);
    if (!idx) return ORA_E_NOMEM;
    int64_t run[ORA_MAXK] = {0};
    for (int64_t ty = 0; ty < GR; ++ty) {
        for (int r = 0; r < K; ++r)
            if ((int64_t)get_u32(rec + row_off + 4 * (ty * K + r)) != run[r]) { free(idx); return ORA_E_RECORD; }
        for (int64_t tx = 0; tx < GC; ++tx) {
            int r = map[ty * GC + tx];
            if (r >= K) { free(idx); return ORA_E_RECORD; }
            idx[ty * GC + tx] = run[r]++;
        }
    }
    for (int r = 0; r < K; ++r)
        if ((int64_t)get_u32(rec + H_COUNT + 4 * r) != run[r]) { free(idx); return ORA_E_RECORD; }
    const int es = dtype_bytes(dtype);
    for (int64_t y = 0; y < M; ++y)
        for (int64_t x = 0; x < N; ++x) {
            const int64_t ty = y / T, tx = x / T;
            const int r = map[ty * GC + tx];
            const int64_t cs = T / b[r];
            const int64_t cy = (y % T) / b[r], cx = (x % T) / b[r];
            const uint64_t cell = (uint64_t)idx[ty * GC + tx] * (uint64_t)(cs * cs) + (uint64_t)(cy * cs + cx);
            for (int64_t ch = 0; ch < C; ++ch) {
                const uint8_t *src = rec + roff[r] + (cell * (uint64_t)C + (uint64_t)ch) * (uint64_t)es;
                if (src + es > rec + len) { free(idx); return ORA_E_RECORD; }
                double v;
                if (dtype == 0) v = (double)get_f32(src);
                else if (dtype == 1) v = (double)*src;
                else /* exact-sum record: the noise-free mean S / b^2 (Eq. 2), in the f32 precision of the means */
                    v = (double)((float)get_u32(src) / (float)(b[r] * b[r]));
                if (out_type == 0) {
                    ((uint8_t *)out)[y * out_pitch + x * C + ch] = (uint8_t)rint(v);
                } else if (out_type == 1) {
                    float *row = (float *)((uint8_t *)out + y * out_pitch);
                    row[x * C + ch] = (float)v;
                } else {
                    double *row = (double *)((uint8_t *)out + y * out_pitch);
                    row[x * C + ch] = v;
                }
            }
        }
    free(idx);
    return ORA_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Differentiable soft layer (training pattern on top of the release; not in the paper).             */
/* y = w * P~_{b0}(x) + (1 - w) * P~_{b1}(x), planar x [B, C, H, W], w [B, 1, H, W], all fp64 here.  */
/* Each P~_b is the uniform release of Alg. 2 (pad, mean, Laplace noise, clip, repeat, crop) with     */
/* R the value range; noise for grid j uses region id j in the counter and frame = frame0 + batch.    */
/* ------------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t B, C, H, W;
    int32_t b[2];
    double eps[2];
    double R, m;
    int32_t pad_mode;
    int32_t noise_free;
    uint32_t stream_id;
    uint64_t seed;
    uint64_t frame0;
} ora_soft_desc;

static int soft_geom(const ora_soft_desc *s, int64_t gr[2], int64_t gc[2], double sigma[2])
{
    if (s->B < 1 || s->C < 1 || s->C > 4 || s->H < 1 || s->W < 1) return ORA_E_INVALID;
    for (int j = 0; j < 2; ++j) {
        if (s->b[j] < 1) return ORA_E_INVALID;
        gr[j] = (s->H + s->b[j] - 1) / s->b[j];
        gc[j] = (s->W + s->b[j] - 1) / s->b[j];
        int64_t pr = gr[j] * s->b[j] - s->H, pc = gc[j] * s->b[j] - s->W;
        int64_t lr = s->pad_mode == 0 ? s->H - 1 : s->H, lc = s->pad_mode == 0 ? s->W - 1 : s->W;
        if (pr > lr || pc > lc) return ORA_E_PAD;
        sigma[j] = s->R * s->m / ((double)s->b[j] * (double)s->b[j] * s->eps[j]);
    }
    return ORA_OK;
}

/* pre_out [B][2][C][gr_j][gc_j] per grid (concatenated: grid 0 block then grid 1 block per image) holds
 * the unclipped noisy means; y_out [B][C][H][W]; p_out [B][2][C][H][W] the broadcast clipped means. */
int ora_soft_forward(const ora_soft_desc *s, const double *x, const double *w, double *y_out, double *p_out)
{
    int64_t gr[2], gc[2];
    double sigma[2];
    int rc = soft_geom(s, gr, gc, sigma);
    if (rc) return rc;
    const int64_t B = s->B, C = s->C, H = s->H, W = s->W;
    for (int64_t n = 0; n < B; ++n)
        for (int j = 0; j < 2; ++j) {
            const int64_t b = s->b[j];
            for (int64_t cy = 0; cy < gr[j]; ++cy)
                for (int64_t cx = 0; cx < gc[j]; ++cx) {
                    uint64_t frame = s->frame0 + (uint64_t)n;
                    uint32_t ctr[4] = {(uint32_t)(cy * gc[j] + cx), (uint32_t)j | (s->stream_id << 8),
                                       (uint32_t)frame, (uint32_t)(frame >> 32)};
                    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
                    uint32_t words[4];
                    ora_philox4x32_10(ctr, key, words);
                    for (int64_t ch = 0; ch < C; ++ch) {
                        const double *plane = x + (n * C + ch) * H * W;
                        double sum = 0.0;
                        for (int64_t y = cy * b; y < (cy + 1) * b; ++y)
                            for (int64_t xx = cx * b; xx < (cx + 1) * b; ++xx)
                                sum += plane[ora_reflect(y, H, s->pad_mode) * W + ora_reflect(xx, W, s->pad_mode)];
                        double eta = s->noise_free ? 0.0 : ora_laplace_from_word(words[ch], sigma[j]);
                        double v = sum / (double)(b * b) + eta;
                        if (v < 0.0) v = 0.0;
                        if (v > s->R) v = s->R;
                        double *pp = p_out + ((n * 2 + j) * C + ch) * H * W;
                        for (int64_t y = cy * b; y < (cy + 1) * b && y < H; ++y)
                            for (int64_t xx = cx * b; xx < (cx + 1) * b && xx < W; ++xx) pp[y * W + xx] = v;
                    }
                }
        }
    for (int64_t n = 0; n < B; ++n)
        for (int64_t ch = 0; ch < C; ++ch)
            for (int64_t i = 0; i < H * W; ++i) {
                double ww = w[n * H * W + i];
                double p0 = p_out[((n * 2 + 0) * C + ch) * H * W + i];
                double p1 = p_out[((n * 2 + 1) * C + ch) * H * W + i];
                y_out[(n * C + ch) * H * W + i] = ww * p0 + (1.0 - ww) * p1;
            }
    return ORA_OK;
}

/*
 * Analytic adjoint of ora_soft_forward for L = sum g * y with the noise held constant:
 *  dL/dw(p) = g(p) * (P~_{b0}(p) - P~_{b1}(p));
 *  dL/dx(q) = sum over grids j, over cells c whose padded samples include q (with multiplicity mult):
 *             [0 < pre_c < R] * mult(q, c) / b_j^2 * sum_{p in c, p inside the image} g(p) * w_j(p),
 *  with w_0 = w and w_1 = 1 - w.  Scattered from every padded sample to its source pixel.
 */
int ora_soft_backward(const ora_soft_desc *s, const double *x, const double *w, const double *g,
                      double *dx, double *dw)
{
    int64_t gr[2], gc[2];
    double sigma[2];
    int rc = soft_geom(s, gr, gc, sigma);
    if (rc) return rc;
    const int64_t B = s->B, C = s->C, H = s->H, W = s->W;
    memset(dx, 0, sizeof(double) * (size_t)(B * C * H * W));
    for (int64_t n = 0; n < B; ++n)
        for (int j = 0; j < 2; ++j) {
            const int64_t b = s->b[j];
            for (int64_t cy = 0; cy < gr[j]; ++cy)
                for (int64_t cx = 0; cx < gc[j]; ++cx) {
                    uint64_t frame = s->frame0 + (uint64_t)n;
                    uint32_t ctr[4] = {(uint32_t)(cy * gc[j] + cx), (uint32_t)j | (s->stream_id << 8),
                                       (uint32_t)frame, (uint32_t)(frame >> 32)};
                    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
                    uint32_t words[4];
                    ora_philox4x32_10(ctr, key, words);
                    for (int64_t ch = 0; ch < C; ++ch) {
                        const double *plane = x + (n * C + ch) * H * W;
                        const double *gp = g + (n * C + ch) * H * W;
                        const double *wp = w + n * H * W;
                        double sum = 0.0, coef = 0.0;
                        for (int64_t y = cy * b; y < (cy + 1) * b; ++y)
                            for (int64_t xx = cx * b; xx < (cx + 1) * b; ++xx) {
                                sum += plane[ora_reflect(y, H, s->pad_mode) * W + ora_reflect(xx, W, s->pad_mode)];
                                if (y < H && xx < W) {
                                    double wj = j == 0 ? wp[y * W + xx] : 1.0 - wp[y * W + xx];
                                    coef += gp[y * W + xx] * wj;
                                }
                            }
                        double eta = s->noise_free ? 0.0 : ora_laplace_from_word(words[ch], sigma[j]);
                        double pre = sum / (double)(b * b) + eta;
                        if (!(pre > 0.0 && pre < s->R)) continue;
                        double per_sample = coef / (double)(b * b);
                        double *dxp = dx + (n * C + ch) * H * W;
                        for (int64_t y = cy * b; y < (cy + 1) * b; ++y)
                            for (int64_t xx = cx * b; xx < (cx + 1) * b; ++xx)
                                dxp[ora_reflect(y, H, s->pad_mode) * W + ora_reflect(xx, W, s->pad_mode)] += per_sample;
                    }
                }
        }
    /* dw from the forward's broadcast means */
    double *y = (double *)malloc(sizeof(double) * (size_t)(B * C * H * W));
    double *p = (double *)malloc(sizeof(double) * (size_t)(B * 2 * C * H * W));
    if (!y || !p) { free(y); free(p); return ORA_E_NOMEM; }
    rc = ora_soft_forward(s, x, w, y, p);
    if (rc) { free(y); free(p); return rc; }
    for (int64_t n = 0; n < B; ++n)
        for (int64_t i = 0; i < H * W; ++i) {
            double acc = 0.0;
            for (int64_t ch = 0; ch < C; ++ch) {
                double p0 = p[((n * 2 + 0) * C + ch) * H * W + i];
                double p1 = p[((n * 2 + 1) * C + ch) * H * W + i];
                acc += g[(n * C + ch) * H * W + i] * (p0 - p1);
            }
            dw[n * H * W + i] = acc;
        }
    free(y);
    free(p);
    return ORA_OK;
}

uint64_t ora_header_size(void) { return H_SIZE; }
