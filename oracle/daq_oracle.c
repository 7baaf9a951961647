/*
 * ORACLE - test infrastructure only.  Plain, slow, obviously correct CPU
 * statement of the muon g-2 DAQ per-fill processing (Sec. 3, Table 2).  Only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may build,
 * load or run it; the CUDA library never does, and the two share no code.
 *
 * Per (fill f, calorimeter c) with crystals x and samples t in [0, len):
 *   1. pedestal   P[x] = floor((sum_{t<n} s[x][t] + floor(n/2)) / n), n = min(ped, len)
 *                 (Table 2, pedestal kernel: average of the first 100 samples,
 *                 rounded half up to an integer ADC count)
 *   2. sum        S[t] = sum_x s[x][t] - sum_x P[x]
 *                 (Table 2, "sum all waveforms" kernel; Sec. 3 Q-method:
 *                 pedestal-subtracted waveform)
 *   3. threshold  A[t] = S[t] > T                (Table 2 threshold kernel; Sec. 3 T-method)
 *   4. windows    M[t] = exists u with A[u] and u - pre <= t <= u + post, t in [0, len)
 *                 (Table 2 pre/post-sample kernel)
 *   5. merge      islands = maximal runs of M (overlapping or touching windows
 *                 become one island) (Table 2 merge kernel)
 *   6. save       island records (fill, calo, start, len, pool_row) in (f, c, start)
 *                 order; pool row r = the raw samples s[x][t] of the r-th marked
 *                 sample (Table 2 save-islands kernel; Sec. 3: islands go back to host)
 *   7. decimate   B_D[k] = sum_{t=kD}^{min(kD+D,len)-1} S[t], k < ceil(len/D)
 *                 (Table 2 Q decimation kernel)
 *   8. fill sum   Q_D[c][k] += B_D[k] over all fills (Table 2 fill-by-fill sum; Sec. 3 Q-method)
 *
 * Step 4 is written as an explicit scan of every window (O(len * (pre+post))),
 * deliberately not the GPU's bit-parallel form.
 *
 * Packed pool stream (lossless; Sec. 3 has the frontend compress island data
 * losslessly before event building, without naming the method - this format
 * is this project's reading):
 *   header   u32 magic 0x50514144, u32 n_xtal, u64 rows
 *   offsets  u64[n_blocks + 1], n_blocks = ceil(rows / 32): byte offset of each
 *            block's payload from the payload start (the last one = its size)
 *   payload  block b = rows [32b, 32b + 32), the last block padded with copies
 *            of the final row; for each crystal x, with v_i the sample of row i
 *            of the block: z_0 = 0, z_i = zigzag(v_i - v_{i-1}),
 *            zigzag(d) = 2d for d >= 0, -2d - 1 for d < 0; w = bit length of
 *            max z_i (0..17); words: (uint16)v_0 | w << 16, then w bit planes,
 *            bit i of plane k = bit k of z_i.
 *
 * Per-crystal full-resolution fill sum (the form Table 2's fill-by-fill sum
 * kernel suggests with one thread per crystal and sample, 54 x 560,000):
 *   Qx[c][x][t] += s[f][c][x][t] - P[f][c][x]   for t < len_f, over all fills f
 *   (pedestal P as in step 1; int64 accumulators).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct oracle_params {
    int32_t threshold, pre, post, ped_samples, n_decim, decim[2];
} oracle_params;

typedef struct oracle_island {
    int32_t fill, calo, start, len;
    int64_t pool_row;
} oracle_island;

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* Step 1 for one crystal row. */
int32_t oracle_pedestal(const int16_t *row, int64_t len, int32_t ped_samples)
{
    int64_t n = ped_samples < len ? ped_samples : len;
    if (n <= 0) return 0;
    int64_t sum = 0;
    for (int64_t t = 0; t < n; ++t) sum += row[t];
    return (int32_t)floor_div(sum + n / 2, n);
}

/*
 * Steps 1-7 for one calorimeter-fill.  s points at [n_xtal][pitch].  Outputs
 * (any may be NULL): ped[n_xtal]; S[len]; mark[len] (M); islands (up to
 * isl_cap, pool_row counted from row_base); pool [rows][n_xtal] (up to
 * row_cap rows, indexed from row 0 = row_base); bins_d[k] for each decimation.
 * Returns island count; *n_rows gets the marked-sample count.
 */
int64_t oracle_calofill(const int16_t *s, int32_t n_xtal, int64_t pitch, int64_t len, const oracle_params *p,
                        int32_t fill, int32_t calo, int32_t *ped, int64_t *S_out, uint8_t *mark_out,
                        oracle_island *isl, int64_t isl_cap, int64_t row_base, int16_t *pool, int64_t row_cap,
                        int64_t *n_rows, int64_t *bins0, int64_t *bins1)
{
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)(len > 0 ? len : 1));
    uint8_t *A = (uint8_t *)malloc((size_t)(len > 0 ? len : 1));
    uint8_t *M = (uint8_t *)malloc((size_t)(len > 0 ? len : 1));

    /* 1. pedestals */
    int64_t ped_total = 0;
    for (int32_t x = 0; x < n_xtal; ++x) {
        int32_t px = oracle_pedestal(s + (int64_t)x * pitch, len, p->ped_samples);
        if (ped) ped[x] = px;
        ped_total += px;
    }
    /* 2. pedestal-subtracted crystal sum */
    for (int64_t t = 0; t < len; ++t) {
        int64_t acc = 0;
        for (int32_t x = 0; x < n_xtal; ++x) acc += s[(int64_t)x * pitch + t];
        S[t] = acc - ped_total;
    }
    /* 3. threshold */
    for (int64_t t = 0; t < len; ++t) A[t] = S[t] > (int64_t)p->threshold;
    /* 4. pre/post windows: t is marked when some crossing u has t in [u - pre, u + post] */
    for (int64_t t = 0; t < len; ++t) {
        int64_t u_lo = t - p->post, u_hi = t + p->pre;
        if (u_lo < 0) u_lo = 0;
        if (u_hi > len - 1) u_hi = len - 1;
        uint8_t m = 0;
        for (int64_t u = u_lo; u <= u_hi; ++u)
            if (A[u]) {
                m = 1;
                break;
            }
        M[t] = m;
    }
    /* 5./6. maximal runs of M, pool rows in time order */
    int64_t n_isl = 0, rows = 0;
    for (int64_t t = 0; t < len; ++t) {
        if (!M[t]) continue;
        if (t == 0 || !M[t - 1]) {
            int64_t e = t;
            while (e + 1 < len && M[e + 1]) ++e;
            if (isl && n_isl < isl_cap) {
                isl[n_isl].fill = fill;
                isl[n_isl].calo = calo;
                isl[n_isl].start = (int32_t)t;
                isl[n_isl].len = (int32_t)(e - t + 1);
                isl[n_isl].pool_row = row_base + rows;
            }
            ++n_isl;
        }
        if (pool && rows < row_cap)
            for (int32_t x = 0; x < n_xtal; ++x) pool[rows * n_xtal + x] = s[(int64_t)x * pitch + t];
        ++rows;
    }
    /* 7. decimation of the pedestal-subtracted sum */
    for (int d = 0; d < p->n_decim; ++d) {
        int64_t D = p->decim[d];
        int64_t *bins = d == 0 ? bins0 : bins1;
        if (!bins) continue;
        for (int64_t k = 0; k * D < len; ++k) {
            int64_t b = 0;
            for (int64_t t = k * D; t < k * D + D && t < len; ++t) b += S[t];
            bins[k] = b;
        }
    }
    if (S_out) memcpy(S_out, S, sizeof(int64_t) * (size_t)len);
    if (mark_out) memcpy(mark_out, M, (size_t)len);
    if (n_rows) *n_rows = rows;
    free(S);
    free(A);
    free(M);
    return n_isl;
}

/*
 * All fills and calorimeters of samples[n_fills][n_calo][n_xtal][pitch], in
 * (fill, calo) order, with step 8 accumulating into q: n_calo rows of
 * ceil(pitch/D0) bins for the first factor, then n_calo rows of ceil(pitch/D1).
 * fill_len may be NULL (every fill is pitch samples long).  Island records and
 * pool rows beyond their capacities are counted but not written; counts[0] =
 * islands, counts[1] = pool rows.  n_threads > 1 runs independent
 * calorimeter-fills on several host threads and then concatenates them in
 * order (results are identical to the single-thread run).  Returns 0, or -1 on
 * bad arguments.
 */
int oracle_process_fills(const int16_t *samples, int32_t n_fills, int32_t n_calo, int32_t n_xtal, int64_t pitch,
                         const int32_t *fill_len, const oracle_params *p, oracle_island *isl, int64_t isl_cap,
                         int16_t *pool, int64_t row_cap, int32_t *ped, int64_t *q, int64_t *counts,
                         int32_t n_threads)
{
    if (!samples || !p || n_fills < 0 || n_calo < 0 || n_xtal <= 0 || pitch < 0 || p->ped_samples <= 0 ||
        p->n_decim < 0 || p->n_decim > 2 || p->pre < 0 || p->post < 0)
        return -1;
    for (int d = 0; d < p->n_decim; ++d)
        if (p->decim[d] <= 0) return -1;
    int64_t nb[2] = {0, 0};
    for (int d = 0; d < p->n_decim; ++d) nb[d] = (pitch + p->decim[d] - 1) / p->decim[d];
    const int64_t n_cf = (int64_t)n_fills * n_calo;

    /* each calorimeter-fill into its own buffers */
    oracle_island **cf_isl = (oracle_island **)calloc((size_t)(n_cf ? n_cf : 1), sizeof(void *));
    int16_t **cf_pool = (int16_t **)calloc((size_t)(n_cf ? n_cf : 1), sizeof(void *));
    int64_t **cf_bins = (int64_t **)calloc((size_t)(n_cf ? n_cf : 1), sizeof(void *));
    int64_t *cf_nisl = (int64_t *)calloc((size_t)(n_cf ? n_cf : 1), sizeof(int64_t));
    int64_t *cf_rows = (int64_t *)calloc((size_t)(n_cf ? n_cf : 1), sizeof(int64_t));
    int64_t *cf_len = (int64_t *)calloc((size_t)(n_cf ? n_cf : 1), sizeof(int64_t));

#ifdef _OPENMP
    if (n_threads > 1) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1) if (n_threads > 1)
#endif
    for (int64_t cf = 0; cf < n_cf; ++cf) {
        int32_t f = (int32_t)(cf / n_calo), c = (int32_t)(cf % n_calo);
        int64_t len = fill_len ? fill_len[f] : pitch;
        if (len < 0) len = 0;
        if (len > pitch) len = pitch;
        cf_len[cf] = len;
        int64_t max_isl = len / 2 + 1;
        cf_isl[cf] = (oracle_island *)malloc(sizeof(oracle_island) * (size_t)max_isl);
        cf_pool[cf] = (int16_t *)malloc(sizeof(int16_t) * (size_t)(len > 0 ? len : 1) * (size_t)n_xtal);
        cf_bins[cf] = (int64_t *)calloc((size_t)(nb[0] + nb[1] + 1), sizeof(int64_t));
        cf_nisl[cf] = oracle_calofill(samples + cf * n_xtal * pitch, n_xtal, pitch, len, p, f, c,
                                      ped ? ped + cf * n_xtal : NULL, NULL, NULL, cf_isl[cf], max_isl, 0,
                                      cf_pool[cf], len, &cf_rows[cf], cf_bins[cf], cf_bins[cf] + nb[0]);
    }

    /* concatenate in (fill, calo) order and accumulate the fill sums */
    int64_t tot_isl = 0, tot_rows = 0;
    for (int64_t cf = 0; cf < n_cf; ++cf) {
        int32_t c = (int32_t)(cf % n_calo);
        for (int64_t i = 0; i < cf_nisl[cf]; ++i) {
            if (isl && tot_isl < isl_cap) {
                isl[tot_isl] = cf_isl[cf][i];
                isl[tot_isl].pool_row += tot_rows;
            }
            ++tot_isl;
        }
        for (int64_t r = 0; r < cf_rows[cf]; ++r) {
            if (pool && tot_rows < row_cap)
                memcpy(pool + tot_rows * n_xtal, cf_pool[cf] + r * n_xtal, sizeof(int16_t) * (size_t)n_xtal);
            ++tot_rows;
        }
        if (q) {
            for (int d = 0; d < p->n_decim; ++d) {
                int64_t kmax = (cf_len[cf] + p->decim[d] - 1) / p->decim[d];
                /* q holds [n_calo][nb[0]] for the first factor, then [n_calo][nb[1]] */
                int64_t *dst = d == 0 ? q + (int64_t)c * nb[0] : q + (int64_t)n_calo * nb[0] + (int64_t)c * nb[1];
                const int64_t *src = cf_bins[cf] + (d == 0 ? 0 : nb[0]);
                for (int64_t k = 0; k < kmax; ++k) dst[k] += src[k];
            }
        }
        free(cf_isl[cf]);
        free(cf_pool[cf]);
        free(cf_bins[cf]);
    }
    if (counts) {
        counts[0] = tot_isl;
        counts[1] = tot_rows;
    }
    free(cf_isl);
    free(cf_pool);
    free(cf_bins);
    free(cf_nisl);
    free(cf_rows);
    free(cf_len);
    return 0;
}

/*
 * Per-crystal full-resolution fill sum: for every fill f, calorimeter c,
 * crystal x and sample t < len_f, add s[f][c][x][t] - P[f][c][x] to
 * q[c][x][t] (int64, layout [n_calo][n_xtal][pitch]; samples past a fill's
 * length add nothing).  fill_len may be NULL (every fill is pitch long).
 */
int oracle_crystal_sum(const int16_t *samples, int32_t n_fills, int32_t n_calo, int32_t n_xtal, int64_t pitch,
                       const int32_t *fill_len, int32_t ped_samples, int64_t *q)
{
    if (n_fills < 0 || n_calo < 0 || n_xtal < 1 || pitch < 0 || ped_samples < 1 || (!q && n_calo > 0)) return -1;
    for (int32_t f = 0; f < n_fills; ++f) {
        int64_t len = fill_len ? fill_len[f] : pitch;
        if (len < 0 || len > pitch) return -1;
        for (int32_t c = 0; c < n_calo; ++c)
            for (int32_t x = 0; x < n_xtal; ++x) {
                const int16_t *row = samples + (((int64_t)f * n_calo + c) * n_xtal + x) * pitch;
                const int64_t ped = oracle_pedestal(row, len, ped_samples);
                int64_t *qrow = q + ((int64_t)c * n_xtal + x) * pitch;
                for (int64_t t = 0; t < len; ++t) qrow[t] += (int64_t)row[t] - ped;
            }
    }
    return 0;
}

/* ---------------------------------------------------------------- packed pool stream */
static void put_u32(uint8_t *p, uint32_t v)
{
    for (int k = 0; k < 4; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

static void put_u64(uint8_t *p, uint64_t v)
{
    for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

static uint32_t get_u32(const uint8_t *p)
{
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k) v |= (uint32_t)p[k] << (8 * k);
    return v;
}

static uint64_t get_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int k = 0; k < 8; ++k) v |= (uint64_t)p[k] << (8 * k);
    return v;
}

static uint32_t zigzag(int32_t d) { return d >= 0 ? 2u * (uint32_t)d : 2u * (uint32_t)(-(int64_t)d) - 1u; }

static int32_t unzigzag(uint32_t z) { return (z & 1u) ? -(int32_t)((z + 1u) / 2u) : (int32_t)(z / 2u); }

static int bit_length(uint32_t v)
{
    int n = 0;
    while (v) {
        ++n;
        v >>= 1;
    }
    return n;
}

/* Block b, crystal x: the 32 samples (padded with the last row). */
static void block_column(const int16_t *pool, int64_t rows, int32_t n_xtal, int64_t b, int32_t x, int32_t v[32])
{
    for (int i = 0; i < 32; ++i) {
        int64_t r = 32 * b + i;
        if (r >= rows) r = rows - 1;
        v[i] = pool[r * n_xtal + x];
    }
}

/* Pack pool[rows][n_xtal]; returns the stream's size, writing only the bytes
 * that fit in cap (out may be NULL with cap 0 to ask for the size). */
int64_t oracle_pack(const int16_t *pool, int64_t rows, int32_t n_xtal, uint8_t *out, int64_t cap)
{
    if (rows < 0 || n_xtal < 1 || cap < 0) return -1;
    const int64_t nb = (rows + 31) / 32;
    const int64_t head = 16 + 8 * (nb + 1);
    int64_t pos = 0; /* payload bytes so far */
    uint8_t w8[8];
#define EMIT(off, nbytes, src)                                                                                   \
    do {                                                                                                         \
        for (int q_ = 0; q_ < (nbytes); ++q_)                                                                    \
            if ((off) + q_ < cap) out[(off) + q_] = (src)[q_];                                                   \
    } while (0)
    put_u32(w8, 0x50514144u);
    put_u32(w8 + 4, (uint32_t)n_xtal);
    EMIT(0, 8, w8);
    put_u64(w8, (uint64_t)rows);
    EMIT(8, 8, w8);
    for (int64_t b = 0; b < nb; ++b) {
        put_u64(w8, (uint64_t)pos);
        EMIT(16 + 8 * b, 8, w8);
        for (int32_t x = 0; x < n_xtal; ++x) {
            int32_t v[32];
            uint32_t z[32];
            block_column(pool, rows, n_xtal, b, x, v);
            uint32_t zmax = 0;
            z[0] = 0;
            for (int i = 1; i < 32; ++i) {
                z[i] = zigzag(v[i] - v[i - 1]);
                if (z[i] > zmax) zmax = z[i];
            }
            const int w = bit_length(zmax);
            put_u32(w8, (uint32_t)(uint16_t)v[0] | ((uint32_t)w << 16));
            EMIT(head + pos, 4, w8);
            pos += 4;
            for (int k = 0; k < w; ++k) {
                uint32_t plane = 0;
                for (int i = 0; i < 32; ++i) plane |= ((z[i] >> k) & 1u) << i;
                put_u32(w8, plane);
                EMIT(head + pos, 4, w8);
                pos += 4;
            }
        }
    }
    put_u64(w8, (uint64_t)pos);
    EMIT(16 + 8 * nb, 8, w8);
#undef EMIT
    return head + pos;
}

/* Unpack a stream into pool_out[rows][n_xtal]; rows and n_xtal must match the
 * header.  Returns 0, or -1 for a malformed stream. */
int oracle_unpack(const uint8_t *in, int64_t bytes, int16_t *pool_out, int64_t rows, int32_t n_xtal)
{
    if (bytes < 16 || get_u32(in) != 0x50514144u || (int32_t)get_u32(in + 4) != n_xtal ||
        (int64_t)get_u64(in + 8) != rows)
        return -1;
    const int64_t nb = (rows + 31) / 32;
    const int64_t head = 16 + 8 * (nb + 1);
    if (bytes < head) return -1;
    for (int64_t b = 0; b < nb; ++b) {
        int64_t pos = head + (int64_t)get_u64(in + 16 + 8 * b);
        for (int32_t x = 0; x < n_xtal; ++x) {
            if (pos + 4 > bytes) return -1;
            const uint32_t h = get_u32(in + pos);
            pos += 4;
            const int w = (int)(h >> 16);
            if (w > 17 || pos + 4 * (int64_t)w > bytes) return -1;
            uint32_t z[32] = {0};
            for (int k = 0; k < w; ++k) {
                const uint32_t plane = get_u32(in + pos);
                pos += 4;
                for (int i = 0; i < 32; ++i) z[i] |= ((plane >> i) & 1u) << k;
            }
            int32_t v = (int16_t)(h & 0xffffu);
            for (int i = 0; i < 32; ++i) {
                if (i > 0) v += unzigzag(z[i]);
                const int64_t r = 32 * b + i;
                if (r < rows) pool_out[r * n_xtal + x] = (int16_t)v;
            }
        }
    }
    return 0;
}
