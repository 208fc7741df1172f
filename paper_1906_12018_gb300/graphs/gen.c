/*
 * Seeded synthetic graph generators for the labeling workloads.
 *
 * This module produces inputs only: it holds none of the labeling method's
 * arithmetic.  Both the GPU path and the CPU oracle are fed from here.
 *
 *   - random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
 *     pseudorandom number generators", OOPSLA 2014) used in counter mode:
 *     draw(seed, stream, i) is output i+1 of the SplitMix64 sequence whose
 *     state starts at a per-(seed, stream) base.  Counter mode makes every
 *     draw independent of thread count, so parallel generation is
 *     deterministic.
 *   - R-MAT (Chakrabarti, Zhan & Faloutsos, SDM 2004): per edge, `scale`
 *     recursive quadrant choices with probabilities (a, b, c, d); no noise,
 *     no id permutation; optional rejection of ids >= n_limit (redrawn).
 *   - Chung-Lu: expected-degree model, both endpoints drawn i.i.d.
 *     proportional to w_i = (i+1)^(-1/(gamma-1)) via a Vose alias table.
 *   - cleaning: symmetrise, drop self-loops and duplicates, sorted CSR.
 *   - largest connected component, renumbered preserving id order.
 *   - degree order: rank -> id, degree descending, ties by smaller id.
 *   - uniform query pairs.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no -march flags;
 * the same source runs on x86-64 and aarch64).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA64 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* base state of the (seed, stream) sequence */
static inline uint64_t stream_base(uint64_t seed, uint64_t stream) {
    return sm64_mix(seed + GAMMA64) ^ sm64_mix(stream * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL);
}

static inline uint64_t draw(uint64_t base, uint64_t i) {
    return sm64_mix(base + (i + 1) * GAMMA64);
}

static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

uint64_t gen_draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return draw(stream_base(seed, stream), i);
}

/* ------------------------------------------------------------------ R-MAT */
/* Writes m edges (src[e], dst[e]).  With n_limit > 0, an edge with either
 * endpoint >= n_limit is redrawn from the next attempt stream.  Returns 0,
 * or -1 if an edge needed more than 4096 attempts. */
int gen_rmat_edges(int scale, int64_t m, double a, double b, double c,
                   uint64_t seed, int64_t n_limit, int32_t* src, int32_t* dst) {
    const double ab = a + b, abc = a + b + c;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int64_t e = 0; e < m; ++e) {
        int ok = 0;
        for (uint64_t attempt = 0; attempt < 4096 && !ok; ++attempt) {
            const uint64_t base = stream_base(seed, attempt);
            uint32_t u = 0, v = 0;
            for (int l = 0; l < scale; ++l) {
                const double r = u01(draw(base, (uint64_t)e * (uint64_t)scale + (uint64_t)l));
                const uint32_t bit = 1u << (scale - 1 - l);
                if (r < a) {
                } else if (r < ab) {
                    v |= bit;
                } else if (r < abc) {
                    u |= bit;
                } else {
                    u |= bit;
                    v |= bit;
                }
            }
            if (n_limit <= 0 || ((int64_t)u < n_limit && (int64_t)v < n_limit)) {
                src[e] = (int32_t)u;
                dst[e] = (int32_t)v;
                ok = 1;
            }
        }
        if (!ok) bad = 1;
    }
    return bad ? -1 : 0;
}

/* -------------------------------------------------------------- Chung-Lu */
/* Both endpoints i.i.d. proportional to w_i = (i+1)^(-1/(gamma-1)).
 * Vose alias table; per endpoint two draws (slot, coin). */
int gen_chung_lu_edges(int64_t n, int64_t m, double gamma, uint64_t seed,
                       int32_t* src, int32_t* dst) {
    if (n <= 0) return -1;
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* alias = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t* small = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* large = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!p || !alias || !small || !large) {
        free(p); free(alias); free(small); free(large);
        return -1;
    }
    const double ex = -1.0 / (gamma - 1.0);
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        p[i] = pow((double)(i + 1), ex);
        sum += p[i];
    }
    /* scaled probabilities p_i * n (mean 1) */
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        p[i] = p[i] / sum * (double)n;
        alias[i] = (int32_t)i;
        if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        const int64_t s = small[--ns];
        const int64_t l = large[nl - 1];
        alias[s] = (int32_t)l;
        p[l] = (p[l] + p[s]) - 1.0;
        if (p[l] < 1.0) {
            --nl;
            small[ns++] = l;
        }
    }
    while (nl > 0) p[large[--nl]] = 1.0;
    while (ns > 0) p[small[--ns]] = 1.0;
    free(small);
    free(large);

    const uint64_t base = stream_base(seed, 1);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int32_t ends[2];
        for (int k = 0; k < 2; ++k) {
            const uint64_t x = draw(base, (uint64_t)e * 4 + (uint64_t)(2 * k));
            const uint64_t y = draw(base, (uint64_t)e * 4 + (uint64_t)(2 * k + 1));
            int64_t slot = (int64_t)(((unsigned __int128)x * (uint64_t)n) >> 64);
            ends[k] = (u01(y) < p[slot]) ? (int32_t)slot : alias[slot];
        }
        src[e] = ends[0];
        dst[e] = ends[1];
    }
    free(p);
    free(alias);
    return 0;
}

/* ---------------------------------------------------- radix sort of keys */
static int bits_for(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

/* LSD radix sort (11-bit digits), parallel histogram + stable scatter. */
static void radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t cnt, int key_bits) {
    enum { RB = 11, RADIX = 1 << RB };
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * (size_t)RADIX * (size_t)nthreads);
    uint64_t* in = keys;
    uint64_t* out = tmp;
    for (int shift = 0; shift < key_bits; shift += RB) {
        memset(hist, 0, sizeof(int64_t) * (size_t)RADIX * (size_t)nthreads);
#pragma omp parallel num_threads(nthreads)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            const int64_t lo = cnt * t / nthreads, hi = cnt * (t + 1) / nthreads;
            int64_t* h = hist + (size_t)t * RADIX;
            for (int64_t i = lo; i < hi; ++i) h[(in[i] >> shift) & (RADIX - 1)]++;
#pragma omp barrier
#pragma omp single
            {
                int64_t run = 0;
                for (int d = 0; d < RADIX; ++d)
                    for (int tt = 0; tt < nthreads; ++tt) {
                        const int64_t c = hist[(size_t)tt * RADIX + d];
                        hist[(size_t)tt * RADIX + d] = run;
                        run += c;
                    }
            }
            for (int64_t i = lo; i < hi; ++i) out[h[(in[i] >> shift) & (RADIX - 1)]++] = in[i];
        }
        uint64_t* s = in;
        in = out;
        out = s;
    }
    if (in != keys) memcpy(keys, in, sizeof(uint64_t) * (size_t)cnt);
    free(hist);
}

/* --------------------------------------------------------------- cleaning */
/* Symmetrise the m input edges over [0,n), drop self-loops and duplicates,
 * and write a CSR with rows sorted ascending.  off must hold n+1 entries,
 * col at least 2m.  Returns the number of arcs (nnz) or -1. */
int64_t gen_clean_csr(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      int64_t* off, int32_t* col) {
    if (n < 0 || m < 0) return -1;
    const int vb = bits_for((uint64_t)(n > 0 ? n - 1 : 0)) ;
    const int sh = vb > 0 ? vb : 1;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    if (!keys || !tmp) {
        free(keys); free(tmp);
        return -1;
    }
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        const uint64_t u = (uint64_t)(uint32_t)src[e], v = (uint64_t)(uint32_t)dst[e];
        if ((int64_t)u >= n || (int64_t)v >= n) {
            free(keys); free(tmp);
            return -1;
        }
        if (u == v) continue;
        keys[k++] = (u << sh) | v;
        keys[k++] = (v << sh) | u;
    }
    radix_sort_u64(keys, tmp, k, 2 * sh);
    free(tmp);
    memset(off, 0, sizeof(int64_t) * (size_t)(n + 1));
    int64_t nnz = 0;
    for (int64_t i = 0; i < k; ++i) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        const int64_t u = (int64_t)(keys[i] >> sh);
        col[nnz++] = (int32_t)(keys[i] & ((1ULL << sh) - 1));
        off[u + 1]++;
    }
    for (int64_t u = 0; u < n; ++u) off[u + 1] += off[u];
    free(keys);
    return nnz;
}

/* ------------------------------------------------------------------- LCC */
/* Largest connected component (ties: the one holding the smallest id).
 * Writes new_id[v] (-1 outside) and returns the component size. */
int64_t gen_lcc_map(int64_t n, const int64_t* off, const int32_t* col, int32_t* new_id) {
    int32_t* comp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) comp[v] = -1;
    int64_t best_size = 0;
    int32_t best = -1, ncomp = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (comp[s] >= 0) continue;
        int64_t h = 0, t = 0;
        q[t++] = (int32_t)s;
        comp[s] = ncomp;
        while (h < t) {
            const int32_t x = q[h++];
            for (int64_t j = off[x]; j < off[x + 1]; ++j) {
                const int32_t y = col[j];
                if (comp[y] < 0) {
                    comp[y] = ncomp;
                    q[t++] = y;
                }
            }
        }
        if (t > best_size) {
            best_size = t;
            best = ncomp;
        }
        ++ncomp;
    }
    int32_t next = 0;
    for (int64_t v = 0; v < n; ++v) new_id[v] = (comp[v] == best) ? next++ : -1;
    free(comp);
    free(q);
    return best_size;
}

/* Induced sub-CSR on the kept vertices (new_id >= 0, monotone in old id,
 * so rows stay sorted).  off_out has n_new+1 entries.  Returns nnz. */
int64_t gen_induce(int64_t n, const int64_t* off, const int32_t* col, const int32_t* new_id,
                   int64_t* off_out, int32_t* col_out) {
    int64_t nnz = 0, r = 0;
    off_out[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (new_id[v] < 0) continue;
        for (int64_t j = off[v]; j < off[v + 1]; ++j) {
            const int32_t y = new_id[col[j]];
            if (y >= 0) col_out[nnz++] = y;
        }
        off_out[++r] = nnz;
    }
    return nnz;
}

/* ---------------------------------------------------------- degree order */
/* order[r] = id of rank r: degree descending, ties by smaller id. */
void gen_degree_order(int64_t n, const int64_t* off, int32_t* order) {
    int64_t maxd = 0;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = off[v + 1] - off[v];
        if (d > maxd) maxd = d;
    }
    int64_t* start = (int64_t*)calloc((size_t)(maxd + 2), sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) start[maxd - (off[v + 1] - off[v])]++;
    int64_t run = 0;
    for (int64_t k = 0; k <= maxd; ++k) {
        const int64_t c = start[k];
        start[k] = run;
        run += c;
    }
    for (int64_t v = 0; v < n; ++v) order[start[maxd - (off[v + 1] - off[v])]++] = (int32_t)v;
    free(start);
}

/* --------------------------------------------------------- query pairs */
/* 2q ints: s_k = pairs[2k], t_k = pairs[2k+1], i.i.d. uniform on [0,n). */
void gen_uniform_pairs(int64_t n, int64_t q, uint64_t seed, int32_t* pairs) {
    const uint64_t base = stream_base(seed, 3);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < 2 * q; ++k) {
        const uint64_t x = draw(base, (uint64_t)k);
        pairs[k] = (int32_t)(((unsigned __int128)x * (uint64_t)n) >> 64);
    }
}

/* log-uniform size 2^U(lo_exp, hi_exp), rounded to nearest */
int64_t gen_log_uniform_size(uint64_t seed, double lo_exp, double hi_exp) {
    const double u = u01(draw(stream_base(seed, 2), 0));
    return (int64_t)llround(exp2(lo_exp + (hi_exp - lo_exp) * u));
}

/* uniform integer in [lo, hi] */
int64_t gen_uniform_int(uint64_t seed, uint64_t stream, uint64_t i, int64_t lo, int64_t hi) {
    const uint64_t x = draw(stream_base(seed, stream), i);
    const uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int64_t)(((unsigned __int128)x * span) >> 64);
}

/* uniform double in [0,1) */
double gen_uniform01(uint64_t seed, uint64_t stream, uint64_t i) {
    return u01(draw(stream_base(seed, stream), i));
}
