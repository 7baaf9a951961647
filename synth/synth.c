/*
 * Seeded synthetic calorimeter waveforms shaped like the muon g-2 fills
 * (Sec. 3: 24 calorimeters of 9x6 PbF2 crystals, 800 MSPS 12-bit digitizers,
 * 700 us fills).  This module is the input generator shared by the oracle and
 * the CUDA path.  It holds none of the method's arithmetic (no pedestal,
 * threshold, island or Q-method step): it only writes int16 samples.
 *
 * Determinism: every random draw is a counter-based SplitMix64 output keyed by
 * (seed, fill, calorimeter, crystal, index), and every transcendental function
 * is computed here from +, -, *, / only (no libm), so the bytes produced are
 * identical on any IEEE-754 host when compiled with -ffp-contract=off.
 *
 * Model (one calorimeter-fill):
 *   sample[x][n] = clamp(ped[x] + noise[x][n] + round(sum_p A_p w_p(x) f(t_n - a_p)), 0, 4095)
 *   - ped[x]: uniform integer in [ped_lo, ped_hi], per (calorimeter, crystal)
 *   - noise: Gaussian of width sigma, rounded to an integer (exact inverse CDF
 *     of the rounded distribution, 32-bit resolution)
 *   - arrivals a_p: inhomogeneous Poisson process with intensity
 *     exp(-t/tau) * (1 + osc_amp * cos(2 pi t / osc_period)), zero before
 *     quiet_samples, scaled so that pulses_per_fill * rate pulses are expected
 *     over nominal_samples; drawn exactly by the time-rescaling construction
 *     (unit-rate exponential gaps mapped through the cumulative intensity)
 *   - f: linear rise over rise_ns, then exp decay with time constant decay_ns
 *   - A_p: log-uniform in [amp_lo, amp_hi], shared over the 3x3 patch around a
 *     uniformly drawn centre crystal with Gaussian weights (profile_sigma in
 *     crystal units), normalised over the patch clipped at the array edge
 *   - samples past a fill's length (inside the row pitch) hold beyond_value.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct synth_config {
    uint64_t seed;
    int32_t n_fills, n_calo, n_rows, n_cols; /* crystals per calorimeter = n_rows * n_cols */
    int64_t n_samples;                       /* row pitch (samples per crystal row) */
    double noise_sigma;                      /* ADC counts per crystal */
    int32_t ped_lo, ped_hi;
    double pulses_per_fill;                  /* expected pulses per calorimeter-fill over nominal_samples */
    double nominal_samples;
    double amp_lo, amp_hi;                   /* ADC counts, summed over the patch */
    double rise_ns, decay_ns, sample_ns;
    double tau_us, osc_period_us, osc_amp;
    double profile_sigma;                    /* crystals */
    int32_t quiet_samples;                   /* no arrivals before this sample */
    int32_t beyond_value;                    /* written in [len, n_samples) */
    int32_t tail_samples;                    /* pulse support after arrival */
    int32_t reserved;
} synth_config;

typedef struct synth_pulse {
    double arrival;   /* in samples, from the fill start */
    double amplitude; /* ADC counts, summed over the patch */
    int32_t centre;   /* crystal index = row * n_cols + col */
    int32_t reserved;
} synth_pulse;

/* ---------------- SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) ---------------- */
#define SM_GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* i-th output of the SplitMix64 sequence whose state starts at key. */
static inline uint64_t sm_at(uint64_t key, uint64_t i) { return sm_mix(key + (i + 1) * SM_GAMMA); }

enum { TAG_PED = 1, TAG_NOISE = 2, TAG_PULSE = 3, TAG_PLAN = 4 };

static uint64_t key_of(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t k = sm_mix(seed + tag * 0xd1b54a32d192ed03ULL);
    k = sm_mix(k + (a + 1) * SM_GAMMA);
    k = sm_mix(k + (b + 1) * 0xa0761d6478bd642fULL);
    k = sm_mix(k + (c + 1) * 0xe7037ed1a0b428dbULL);
    return k;
}

static inline double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

/* ---------------- elementary functions from basic arithmetic ---------------- */
static const double D_LN2 = 0.69314718055994530942;
static const double D_LN2_HI = 0.693145751953125; /* 16 significant bits: k*hi is exact */
static const double D_LN2_LO = 1.42860682030941723212e-6;
static const double D_PI = 3.14159265358979323846;

/* exp(x): x = k ln2 + r, |r| <= ln2/2, Taylor series of degree 17, times 2^k. */
static double d_exp(double x)
{
    if (x < -740.0) return 0.0;
    double kf = floor(x / D_LN2 + 0.5);
    double r = (x - kf * D_LN2_HI) - kf * D_LN2_LO;
    double p = 1.0;
    for (int n = 17; n >= 1; --n) p = 1.0 + p * r / (double)n;
    return ldexp(p, (int)kf);
}

/* log(x), x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)), log m = 2 atanh((m-1)/(m+1)). */
static double d_log(double x)
{
    int e;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) {
        m *= 2.0;
        e -= 1;
    }
    double s = (m - 1.0) / (m + 1.0), s2 = s * s, term = s, sum = 0.0;
    for (int n = 1; n <= 41; n += 2) {
        sum += term / (double)n;
        term *= s2;
    }
    return (double)e * D_LN2_HI + ((double)e * D_LN2_LO + 2.0 * sum);
}

/* cos(x): reduce to |r| <= pi, Taylor series in r^2 up to r^36. */
static double d_cos(double x)
{
    const double two_pi_hi = 6.28318530717958623200, two_pi_lo = 2.44929359829470635446e-16;
    double k = floor(x / (2.0 * D_PI) + 0.5);
    double r = (x - k * two_pi_hi) - k * two_pi_lo, r2 = r * r;
    double p = 1.0;
    for (int n = 36; n >= 2; n -= 2) p = 1.0 - p * r2 / ((double)n * (double)(n - 1));
    return p;
}

/* Standard normal CDF by composite Simpson integration of the density from -12. */
static double d_phi(double z)
{
    const double lo = -12.0;
    if (z <= lo) return 0.0;
    int n = 2 * (int)ceil((z - lo) * 400.0);
    double h = (z - lo) / n, acc = 0.0;
    for (int i = 0; i <= n; ++i) {
        double x = lo + h * i;
        double w = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        acc += w * d_exp(-0.5 * x * x);
    }
    return acc * h / 3.0 / 2.50662827463100050242; /* sqrt(2 pi) */
}

/* ---------------- rounded-Gaussian noise by exact inverse CDF ---------------- */
typedef struct noise_table {
    int k_max;          /* values in [-k_max, k_max] */
    uint64_t *thr;      /* thr[i]: P(value <= i - k_max) * 2^32, last = 2^32 */
    int32_t guide[1024];
} noise_table;

static void noise_table_init(noise_table *nt, double sigma)
{
    nt->k_max = sigma > 0 ? (int)ceil(8.0 * sigma) + 1 : 0;
    int n = 2 * nt->k_max + 1;
    nt->thr = (uint64_t *)malloc(sizeof(uint64_t) * n);
    for (int i = 0; i < n; ++i) {
        int k = i - nt->k_max;
        if (i == n - 1 || sigma <= 0) {
            nt->thr[i] = 1ULL << 32;
        } else {
            double c = d_phi((k + 0.5) / sigma) * 4294967296.0;
            nt->thr[i] = (uint64_t)floor(c);
        }
    }
    if (sigma <= 0)
        for (int i = 0; i < n; ++i) nt->thr[i] = 1ULL << 32;
    int k = 0;
    for (int g = 0; g < 1024; ++g) {
        uint64_t v = (uint64_t)g << 22;
        while (nt->thr[k] <= v) ++k;
        nt->guide[g] = k;
    }
}

static inline int noise_draw(const noise_table *nt, uint32_t v)
{
    int k = nt->guide[v >> 22];
    while ((uint64_t)v >= nt->thr[k]) ++k;
    return k - nt->k_max;
}

/* ---------------- pulse arrivals ---------------- */
/* cum[n] = integral of the (unscaled) intensity over samples [0, n). */
static double *intensity_cumulative(const synth_config *cfg, int64_t n_max)
{
    double *cum = (double *)malloc(sizeof(double) * (size_t)(n_max + 1));
    double acc = 0.0;
    const double ns_to_us = 1e-3;
    for (int64_t n = 0; n < n_max; ++n) {
        cum[n] = acc;
        double lam = 0.0;
        if (n >= cfg->quiet_samples) {
            double t_us = (double)n * cfg->sample_ns * ns_to_us;
            lam = d_exp(-t_us / cfg->tau_us) *
                  (1.0 + cfg->osc_amp * d_cos(2.0 * D_PI * t_us / cfg->osc_period_us));
        }
        acc += lam;
    }
    cum[n_max] = acc;
    return cum;
}

static int64_t draw_pulses(const synth_config *cfg, const double *cum, int64_t cum_len, int fill, int calo,
                           int64_t len, double rate, synth_pulse *out, int64_t cap)
{
    int64_t nominal = (int64_t)cfg->nominal_samples;
    if (nominal > cum_len) nominal = cum_len;
    double norm = cum[nominal];
    if (norm <= 0 || rate <= 0 || cfg->pulses_per_fill <= 0 || len <= 0) return 0;
    double scale = cfg->pulses_per_fill * rate / norm; /* pulses per unit of cum */
    double end = cum[len];
    int n_x = cfg->n_rows * cfg->n_cols;
    uint64_t key = key_of(cfg->seed, TAG_PULSE, (uint64_t)fill, (uint64_t)calo, 0);
    double target = 0.0;
    int64_t count = 0, lo = 0;
    for (uint64_t i = 0;; i += 3) {
        double u = u01(sm_at(key, i));
        target += -d_log(1.0 - u) / scale;
        if (target >= end) break;
        /* smallest n with cum[n + 1] > target */
        int64_t a = lo, b = len - 1;
        while (a < b) {
            int64_t mid = a + (b - a) / 2;
            if (cum[mid + 1] > target)
                b = mid;
            else
                a = mid + 1;
        }
        lo = a;
        double width = cum[a + 1] - cum[a];
        double phase = width > 0 ? (target - cum[a]) / width : 0.0;
        if (count < cap) {
            double ua = u01(sm_at(key, i + 1));
            uint64_t uc = sm_at(key, i + 2);
            out[count].arrival = (double)a + phase;
            out[count].amplitude = cfg->amp_lo * d_exp(ua * d_log(cfg->amp_hi / cfg->amp_lo));
            out[count].centre = (int32_t)((uc >> 11) % (uint64_t)n_x);
            out[count].reserved = 0;
        }
        ++count;
    }
    return count;
}

static double pulse_shape(const synth_config *cfg, double dt_ns)
{
    if (dt_ns < 0) return 0.0;
    if (dt_ns < cfg->rise_ns) return dt_ns / cfg->rise_ns;
    return d_exp(-(dt_ns - cfg->rise_ns) / cfg->decay_ns);
}

/* ---------------- one calorimeter-fill ---------------- */
static void render_calofill(const synth_config *cfg, const noise_table *nt, const double *cum, int64_t cum_len,
                            int fill, int calo, int64_t len, double rate, int16_t *out /* [X][pitch] */,
                            double *sig /* [pitch], zeroed */)
{
    const int n_x = cfg->n_rows * cfg->n_cols;
    const int64_t pitch = cfg->n_samples;
    if (len > pitch) len = pitch;
    int64_t n_p = draw_pulses(cfg, cum, cum_len, fill, calo, len, rate, NULL, 0);
    synth_pulse *pl = (synth_pulse *)malloc(sizeof(synth_pulse) * (size_t)(n_p > 0 ? n_p : 1));
    draw_pulses(cfg, cum, cum_len, fill, calo, len, rate, pl, n_p);

    /* patch normalisation for every centre */
    double *norm = (double *)malloc(sizeof(double) * n_x);
    for (int cc = 0; cc < n_x; ++cc) {
        int r0 = cc / cfg->n_cols, c0 = cc % cfg->n_cols;
        double s = 0;
        for (int dr = -1; dr <= 1; ++dr)
            for (int dc = -1; dc <= 1; ++dc) {
                int r = r0 + dr, c = c0 + dc;
                if (r < 0 || r >= cfg->n_rows || c < 0 || c >= cfg->n_cols) continue;
                s += d_exp(-(double)(dr * dr + dc * dc) / (2.0 * cfg->profile_sigma * cfg->profile_sigma));
            }
        norm[cc] = s;
    }

    for (int x = 0; x < n_x; ++x) {
        int r = x / cfg->n_cols, c = x % cfg->n_cols;
        /* pulse signal on this crystal */
        for (int64_t p = 0; p < n_p; ++p) {
            int r0 = pl[p].centre / cfg->n_cols, c0 = pl[p].centre % cfg->n_cols;
            int dr = r - r0, dc = c - c0;
            if (dr < -1 || dr > 1 || dc < -1 || dc > 1) continue;
            double w = d_exp(-(double)(dr * dr + dc * dc) / (2.0 * cfg->profile_sigma * cfg->profile_sigma)) /
                       norm[pl[p].centre];
            double amp = pl[p].amplitude * w;
            int64_t n0 = (int64_t)ceil(pl[p].arrival);
            for (int64_t n = n0; n < n0 + cfg->tail_samples && n < len; ++n)
                sig[n] += amp * pulse_shape(cfg, ((double)n - pl[p].arrival) * cfg->sample_ns);
        }
        uint64_t pk = key_of(cfg->seed, TAG_PED, (uint64_t)calo, (uint64_t)x, 0);
        int ped = cfg->ped_lo + (int)(sm_at(pk, 0) % (uint64_t)(cfg->ped_hi - cfg->ped_lo + 1));
        uint64_t nk = key_of(cfg->seed, TAG_NOISE, (uint64_t)fill, (uint64_t)calo, (uint64_t)x);
        int16_t *row = out + (int64_t)x * pitch;
        for (int64_t n = 0; n < len; ++n) {
            uint64_t z = sm_at(nk, (uint64_t)(n >> 1));
            uint32_t v = (n & 1) ? (uint32_t)(z >> 32) : (uint32_t)z;
            int64_t val = ped + noise_draw(nt, v) + (int64_t)floor(sig[n] + 0.5);
            if (val < 0) val = 0;
            if (val > 4095) val = 4095;
            row[n] = (int16_t)val;
        }
        for (int64_t n = len; n < pitch; ++n) row[n] = (int16_t)cfg->beyond_value;
        /* clear the touched signal samples */
        for (int64_t p = 0; p < n_p; ++p) {
            int64_t n0 = (int64_t)ceil(pl[p].arrival);
            for (int64_t n = n0; n < n0 + cfg->tail_samples && n < len; ++n) sig[n] = 0.0;
        }
    }
    free(norm);
    free(pl);
}

/* Per-fill lengths (uniform integer in [len_lo, len_hi]) and pulse-rate factors
 * (log-uniform in [rate_lo, rate_hi]) for a batch of uneven fills. */
int synth_fill_plan(uint64_t seed, int32_t n_fills, int64_t len_lo, int64_t len_hi, double rate_lo,
                    double rate_hi, int32_t *len_out, double *rate_out)
{
    if (n_fills < 0 || len_lo > len_hi || rate_lo <= 0 || rate_hi < rate_lo) return -1;
    uint64_t key = key_of(seed, TAG_PLAN, 0, 0, 0);
    for (int f = 0; f < n_fills; ++f) {
        uint64_t a = sm_at(key, 2 * (uint64_t)f), b = sm_at(key, 2 * (uint64_t)f + 1);
        if (len_out) len_out[f] = (int32_t)(len_lo + (int64_t)((a >> 11) % (uint64_t)(len_hi - len_lo + 1)));
        if (rate_out) rate_out[f] = rate_lo * d_exp(u01(b) * d_log(rate_hi / rate_lo));
    }
    return 0;
}

/* Fill out[n][C][X][n_samples] with fills [f0, f0 + n) of the configuration
 * (bytes identical to those fills in a whole-batch call).  fill_len / rate are
 * indexed by the absolute fill and may be NULL (all n_samples / 1.0). */
int synth_generate_fills(const synth_config *cfg, int32_t f0, int32_t n, const int32_t *fill_len,
                         const double *rate, int16_t *out, int n_threads)
{
    if (!cfg || !out || cfg->n_fills < 0 || cfg->n_calo < 0 || cfg->n_rows <= 0 || cfg->n_cols <= 0 ||
        cfg->n_samples < 0 || cfg->ped_hi < cfg->ped_lo || f0 < 0 || n < 0 || f0 + n > cfg->n_fills)
        return -1;
    const int64_t n_x = (int64_t)cfg->n_rows * cfg->n_cols, pitch = cfg->n_samples;
    int64_t cum_len = pitch > (int64_t)cfg->nominal_samples ? pitch : (int64_t)cfg->nominal_samples;
    double *cum = intensity_cumulative(cfg, cum_len);
    noise_table nt;
    noise_table_init(&nt, cfg->noise_sigma);
    const int64_t n_cf = (int64_t)n * cfg->n_calo;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double *sig = (double *)calloc((size_t)(pitch > 0 ? pitch : 1), sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t cf = 0; cf < n_cf; ++cf) {
            int f = f0 + (int)(cf / cfg->n_calo), c = (int)(cf % cfg->n_calo);
            int64_t len = fill_len ? fill_len[f] : pitch;
            if (len < 0) len = 0;
            if (len > pitch) len = pitch;
            double rt = rate ? rate[f] : 1.0;
            render_calofill(cfg, &nt, cum, cum_len, f, c, len, rt, out + cf * n_x * pitch, sig);
        }
        free(sig);
    }
    free(nt.thr);
    free(cum);
    return 0;
}

/* Fill out[F][C][X][n_samples].  fill_len / rate may be NULL (all n_samples / 1.0). */
int synth_generate(const synth_config *cfg, const int32_t *fill_len, const double *rate, int16_t *out,
                   int n_threads)
{
    if (!cfg) return -1;
    return synth_generate_fills(cfg, 0, cfg->n_fills, fill_len, rate, out, n_threads);
}

/* Truth list of one calorimeter-fill, in arrival order.  Returns the pulse
 * count (entries beyond cap are not written). */
int64_t synth_pulses(const synth_config *cfg, int32_t fill, int32_t calo, int64_t len, double rate,
                     synth_pulse *out, int64_t cap)
{
    int64_t cum_len = cfg->n_samples > (int64_t)cfg->nominal_samples ? cfg->n_samples : (int64_t)cfg->nominal_samples;
    if (len > cfg->n_samples) len = cfg->n_samples;
    double *cum = intensity_cumulative(cfg, cum_len);
    int64_t n = draw_pulses(cfg, cum, cum_len, fill, calo, len, rate, out, cap);
    free(cum);
    return n;
}

/* True pedestal of (calo, crystal) as drawn by the generator. */
int32_t synth_true_pedestal(const synth_config *cfg, int32_t calo, int32_t xtal)
{
    uint64_t pk = key_of(cfg->seed, TAG_PED, (uint64_t)calo, (uint64_t)xtal, 0);
    return cfg->ped_lo + (int32_t)(sm_at(pk, 0) % (uint64_t)(cfg->ped_hi - cfg->ped_lo + 1));
}

/* Self-check hooks for the elementary functions (tests compare them to libm). */
double synth_exp(double x) { return d_exp(x); }
double synth_log(double x) { return d_log(x); }
double synth_cos(double x) { return d_cos(x); }
double synth_phi(double z) { return d_phi(z); }
int synth_noise_hist(double sigma, uint64_t seed, int64_t n, int64_t *hist, int k_max)
{
    noise_table nt;
    noise_table_init(&nt, sigma);
    uint64_t key = key_of(seed, TAG_NOISE, 0, 0, 0);
    for (int64_t i = 0; i < n; ++i) {
        int v = noise_draw(&nt, (uint32_t)sm_at(key, (uint64_t)i));
        if (v < -k_max) v = -k_max;
        if (v > k_max) v = k_max;
        hist[v + k_max]++;
    }
    free(nt.thr);
    return 0;
}
