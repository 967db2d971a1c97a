/*
 * synth.c -- seeded synthetic inputs for the correction loop.
 *
 * This module only makes inputs.  It holds none of the correction method's
 * arithmetic; both the CPU oracle and the CUDA path read what it writes.
 * Every generator is deterministic for a given seed and independent of the
 * number of OpenMP threads: each value is a pure function of (seed, index),
 * drawn from a counter-based generator, and every sum runs in a fixed order.
 *
 * Generators (all computed in double precision, stored as float32):
 *   - fractal Perlin gradient noise (Perlin's 2002 "improved noise":
 *     Fisher-Yates permutation of 0..255, quintic fade 6t^5-15t^4+10t^3,
 *     twelve edge-direction gradients picked by the hash), summed over
 *     octaves with lacunarity 2 and gain 0.5, min-max scaled to [0,1];
 *   - a Gaussian-peak field: iid Poisson(lambda) counts per voxel plus
 *     isotropic Gaussians (centre uniform in the domain, sigma ~ U[1.5,6],
 *     amplitude ~ LogNormal(0,1), cut at 4 sigma), min-max scaled to [0,1];
 *   - two stand-ins for a lossy compressor's output fhat: uniform noise in
 *     [-xi, xi], and uniform scalar quantization with bin width 2 xi
 *     (fhat = 2 xi * round(f / 2 xi), as a prediction-free SZ-style
 *     quantizer would give).  A value that float32 rounding would push past
 *     the bound is moved toward f one ulp at a time.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden gamma,
 * output is the mixed state.  syn_rand(key, i) is the (i+1)-th output of the
 * stream started at key, so any element can be drawn on its own. */
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static const uint64_t GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t syn_rand(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GAMMA); }

/* uniform double in [0, 1) with 53 random bits */
static double u01(uint64_t key, uint64_t i) { return (double)(syn_rand(key, i) >> 11) * 0x1.0p-53; }

static uint64_t stream_key(uint64_t seed, uint64_t stream) { return mix64(seed * 0xD1B54A32D192ED03ULL + stream); }

/* ---------------------------------------------------------------- Perlin */
typedef struct { int p[512]; } perm_t;

static void make_perm(perm_t *pt, uint64_t key)
{
    int a[256];
    for (int i = 0; i < 256; ++i) a[i] = i;
    for (int i = 255; i > 0; --i) {           /* Fisher-Yates */
        int j = (int)(syn_rand(key, (uint64_t)i) % (uint64_t)(i + 1));
        int t = a[i]; a[i] = a[j]; a[j] = t;
    }
    for (int i = 0; i < 512; ++i) pt->p[i] = a[i & 255];
}

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }
static double lerp(double t, double a, double b) { return a + t * (b - a); }

/* dot product of (x,y,z) with one of the 12 cube-edge directions */
static double grad(int h, double x, double y, double z)
{
    h &= 15;
    double u = h < 8 ? x : y;
    double v = h < 4 ? y : ((h == 12 || h == 14) ? x : z);
    return ((h & 1) ? -u : u) + ((h & 2) ? -v : v);
}

static double noise3(const perm_t *pt, double x, double y, double z)
{
    const int *p = pt->p;
    double fx = floor(x), fy = floor(y), fz = floor(z);
    int X = (int)fx & 255, Y = (int)fy & 255, Z = (int)fz & 255;
    x -= fx; y -= fy; z -= fz;
    double u = fade(x), v = fade(y), w = fade(z);
    int A = p[X] + Y, AA = p[A] + Z, AB = p[A + 1] + Z;
    int B = p[X + 1] + Y, BA = p[B] + Z, BB = p[B + 1] + Z;
    return lerp(w, lerp(v, lerp(u, grad(p[AA], x, y, z), grad(p[BA], x - 1, y, z)),
                           lerp(u, grad(p[AB], x, y - 1, z), grad(p[BB], x - 1, y - 1, z))),
                   lerp(v, lerp(u, grad(p[AA + 1], x, y, z - 1), grad(p[BA + 1], x - 1, y, z - 1)),
                           lerp(u, grad(p[AB + 1], x, y - 1, z - 1), grad(p[BB + 1], x - 1, y - 1, z - 1))));
}

static void minmax_f(const float *v, int64_t n, float *mn, float *mx)
{
    float lo = v[0], hi = v[0];
#pragma omp parallel for reduction(min : lo) reduction(max : hi) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (v[i] < lo) lo = v[i];
        if (v[i] > hi) hi = v[i];
    }
    *mn = lo;
    *mx = hi;
}

static void rescale01(float *v, int64_t n)
{
    float lo, hi;
    minmax_f(v, n, &lo, &hi);
    double d = (double)hi - (double)lo;
    if (!(d > 0)) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) v[i] = 0.0f;
        return;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) v[i] = (float)(((double)v[i] - (double)lo) / d);
}

/* Fractal Perlin noise on an nx*ny*nz grid (nz = 1 for 2D), x fastest.
 * period = lattice spacing of the first octave in voxels. */
void syn_perlin(float *out, int64_t nx, int64_t ny, int64_t nz, int octaves, double period, uint64_t seed)
{
    perm_t pt;
    make_perm(&pt, stream_key(seed, 1));
    double off[32][3];
    if (octaves > 32) octaves = 32;
    for (int o = 0; o < octaves; ++o)
        for (int c = 0; c < 3; ++c) off[o][c] = 256.0 * u01(stream_key(seed, 2), (uint64_t)(3 * o + c));
    int64_t plane = nx * ny;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y) {
            for (int64_t x = 0; x < nx; ++x) {
                double s = 0.0, amp = 1.0, scale = 1.0 / period;
                for (int o = 0; o < octaves; ++o) {
                    s += amp * noise3(&pt, (x + 0.5) * scale + off[o][0], (y + 0.5) * scale + off[o][1],
                                      (z + 0.5) * scale + off[o][2]);
                    amp *= 0.5;
                    scale *= 2.0;
                }
                out[x + nx * y + plane * z] = (float)s;
            }
        }
    rescale01(out, plane * nz);
}

/* ----------------------------------------------------------- Gaussian peaks */
static int poisson_knuth(double lambda, uint64_t key, uint64_t base)
{
    double L = exp(-lambda), p = 1.0;
    int k = 0;
    do {
        ++k;
        p *= u01(key, base + (uint64_t)k);
    } while (p > L && k < 63);
    return k - 1;
}

void syn_peaks(float *out, int64_t nx, int64_t ny, int64_t nz, int64_t npeaks, double lambda, uint64_t seed)
{
    uint64_t kb = stream_key(seed, 10), kp = stream_key(seed, 11);
    int64_t plane = nx * ny;
    double *cx = malloc(sizeof(double) * (size_t)(npeaks > 0 ? npeaks : 1));
    double *cy = malloc(sizeof(double) * (size_t)(npeaks > 0 ? npeaks : 1));
    double *cz = malloc(sizeof(double) * (size_t)(npeaks > 0 ? npeaks : 1));
    double *sg = malloc(sizeof(double) * (size_t)(npeaks > 0 ? npeaks : 1));
    double *am = malloc(sizeof(double) * (size_t)(npeaks > 0 ? npeaks : 1));
    for (int64_t p = 0; p < npeaks; ++p) {
        uint64_t b = (uint64_t)p * 8;
        cx[p] = u01(kp, b + 0) * (double)nx;
        cy[p] = u01(kp, b + 1) * (double)ny;
        cz[p] = u01(kp, b + 2) * (double)nz;
        sg[p] = 1.5 + 4.5 * u01(kp, b + 3);
        double u1 = u01(kp, b + 4), u2 = u01(kp, b + 5);   /* Box-Muller */
        double gauss = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586476925 * u2);
        am[p] = exp(gauss);
    }
#pragma omp parallel
    {
        double *acc = malloc(sizeof(double) * (size_t)plane);
#pragma omp for schedule(dynamic, 1)
        for (int64_t z = 0; z < nz; ++z) {
            for (int64_t q = 0; q < plane; ++q)
                acc[q] = (double)poisson_knuth(lambda, kb, (uint64_t)(z * plane + q) * 64);
            for (int64_t p = 0; p < npeaks; ++p) {   /* fixed order: peak index */
                double r = 4.0 * sg[p], dz = (double)z - cz[p];
                if (fabs(dz) > r) continue;
                double inv = 1.0 / (2.0 * sg[p] * sg[p]);
                int64_t y0 = (int64_t)ceil(cy[p] - r), y1 = (int64_t)floor(cy[p] + r);
                int64_t x0 = (int64_t)ceil(cx[p] - r), x1 = (int64_t)floor(cx[p] + r);
                if (y0 < 0) y0 = 0;
                if (x0 < 0) x0 = 0;
                if (y1 > ny - 1) y1 = ny - 1;
                if (x1 > nx - 1) x1 = nx - 1;
                for (int64_t y = y0; y <= y1; ++y) {
                    double dy = (double)y - cy[p];
                    for (int64_t x = x0; x <= x1; ++x) {
                        double dx = (double)x - cx[p];
                        double d2 = dx * dx + dy * dy + dz * dz;
                        if (d2 > r * r) continue;
                        acc[x + nx * y] += am[p] * exp(-d2 * inv);
                    }
                }
            }
            for (int64_t q = 0; q < plane; ++q) out[z * plane + q] = (float)acc[q];
        }
        free(acc);
    }
    free(cx); free(cy); free(cz); free(sg); free(am);
    rescale01(out, plane * nz);
}

/* ------------------------------------------------- compressor stand-ins */
/* Conservative bound test with a margin far above double rounding error:
 * true |a - b| <= xi whenever this returns 1. */
static int safely_within(float a, float b, float xi)
{
    double d = fabs((double)a - (double)b);
    return d <= (double)xi * (1.0 - 0x1.0p-20);
}

static float pull_inside(float fh, float f, float xi)
{
    int guard = 0;
    while (!safely_within(fh, f, xi) && guard++ < 1 << 20) fh = nextafterf(fh, f);
    return safely_within(fh, f, xi) ? fh : f;
}

void syn_perturb_uniform(const float *f, float *fhat, int64_t n, float xi, uint64_t seed)
{
    uint64_t key = stream_key(seed, 20);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double u = 2.0 * u01(key, (uint64_t)i) - 1.0;
        float fh = (float)((double)f[i] + u * (double)xi);
        fhat[i] = pull_inside(fh, f[i], xi);
    }
}

void syn_prequantize(const float *f, float *fhat, int64_t n, float xi)
{
    double w = 2.0 * (double)xi;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float fh = w > 0 ? (float)(w * nearbyint((double)f[i] / w)) : f[i];
        fhat[i] = pull_inside(fh, f[i], xi);
    }
}

void syn_minmax(const float *v, int64_t n, float *mn, float *mx) { minmax_f(v, n, mn, mx); }

/* Fill out[0..n) with uniform doubles in [0,1) from stream (seed, stream). */
void syn_uniform(double *out, int64_t n, uint64_t seed, uint64_t stream)
{
    uint64_t key = stream_key(seed, 100 + stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = u01(key, (uint64_t)i);
}

int syn_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
