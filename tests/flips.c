/*
 * Test helper (not part of the oracle): which Gaussians two projections of
 * the same scene composite differently.  For every pixel it walks a tile list
 * with the compositing decisions (alpha = min(0.99, o exp(P)), skipped below
 * 1/255, stop before T would drop under 1e-4) in double precision, and flags
 * each Gaussian kept under one projection and not the other.  The parity
 * tests use it to find the Gaussians whose float32 and float64 decisions sit
 * on a threshold, so that they can be left out of a comparison: it decides
 * where two correct results may differ and computes no expected value.
 *
 * proj records [V][n][16] (u, v, depth, opacity, A, B, C, ...), lists and
 * ranges [T][2] per tile; views given by width / height, tile size `tile`.
 *
 * decision_margins() gives, per pixel, how close the decisions of its walk
 * come to their thresholds, so that a test can tell a contributor count that
 * two precisions may decide differently from a wrong one.  same_sequences()
 * marks the pixels whose kept fragments two projections composite in the
 * same order: two depths within rounding of each other may be sorted either
 * way, which changes the pixel without either result being wrong.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int kept(const double* proj, int64_t vn, const uint32_t* vals, uint32_t s, uint32_t e, double px,
                double py, uint32_t* out) {
    double T = 1.0;
    int m = 0;
    for (uint32_t j = s; j < e; ++j) {
        const double* o = proj + (vn + vals[j]) * 16;
        double dx = o[0] - px, dy = o[1] - py;
        double P = -0.5 * (o[4] * dx * dx + o[6] * dy * dy) - o[5] * dx * dy;
        if (P > 0.0) continue;
        double al = fmin(0.99, o[3] * exp(P));
        if (al < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - al);
        if (Tn < 1e-4) break;
        out[m++] = vals[j];
        T = Tn;
    }
    return m;
}

static int by_value(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int64_t flips(int V, int64_t n, const int32_t* width, const int32_t* height, int tile, const double* projA,
              const uint32_t* valsA, const uint32_t* rangesA, const double* projB, const uint32_t* valsB,
              const uint32_t* rangesB, uint8_t* flags) {
    memset(flags, 0, (size_t)V * (size_t)n);
    int64_t npix = 0, toff = 0;
    for (int v = 0; v < V; ++v) {
        int W = width[v], H = height[v], TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
        int64_t vn = (int64_t)v * n;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int64_t t = toff + (int64_t)(y / tile) * TX + x / tile;
                uint32_t la = rangesA[2 * t + 1] - rangesA[2 * t], lb = rangesB[2 * t + 1] - rangesB[2 * t];
                uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * (la + 1));
                uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * (lb + 1));
                int ma = kept(projA, vn, valsA, rangesA[2 * t], rangesA[2 * t + 1], x + 0.5, y + 0.5, A);
                int mb = kept(projB, vn, valsB, rangesB[2 * t], rangesB[2 * t + 1], x + 0.5, y + 0.5, B);
                qsort(A, (size_t)ma, sizeof(uint32_t), by_value);
                qsort(B, (size_t)mb, sizeof(uint32_t), by_value);
                int i = 0, k = 0, differ = 0;
                while (i < ma || k < mb) {
                    if (k >= mb || (i < ma && A[i] < B[k])) { flags[vn + A[i]] = 1; ++i; differ = 1; }
                    else if (i >= ma || B[k] < A[i]) { flags[vn + B[k]] = 1; ++k; differ = 1; }
                    else { ++i; ++k; }
                }
                npix += differ;
                free(A);
                free(B);
            }
        toff += (int64_t)TX * TY;
    }
    return npix;
}

/* Per pixel (views concatenated, row-major), the smallest distance from its
 * threshold of any decision the double-precision walk of its list takes, up
 * to and including the fragment that ends it: the sign test of P (|P|), the
 * alpha cut-off (|255 o e^P - 1|) and the termination test
 * (|T (1 - alpha) / 1e-4 - 1|), each relative to its threshold's scale.
 * Pixels whose list is empty get 1e300. */
void decision_margins(int V, int64_t n, const int32_t* width, const int32_t* height, int tile,
                      const double* proj, const uint32_t* vals, const uint32_t* ranges, double* margin) {
    int64_t toff = 0, poff = 0;
    for (int v = 0; v < V; ++v) {
        int W = width[v], H = height[v], TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
        int64_t vn = (int64_t)v * n;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int64_t t = toff + (int64_t)(y / tile) * TX + x / tile;
                double px = x + 0.5, py = y + 0.5, T = 1.0, m = 1e300;
                for (uint32_t j = ranges[2 * t]; j < ranges[2 * t + 1]; ++j) {
                    const double* o = proj + (vn + vals[j]) * 16;
                    double dx = o[0] - px, dy = o[1] - py;
                    double P = -0.5 * (o[4] * dx * dx + o[6] * dy * dy) - o[5] * dx * dy;
                    m = fmin(m, fabs(P));
                    if (P > 0.0) continue;
                    double raw = o[3] * exp(P);
                    m = fmin(m, fabs(255.0 * raw - 1.0));
                    double al = fmin(0.99, raw);
                    if (al < 1.0 / 255.0) continue;
                    double Tn = T * (1.0 - al);
                    m = fmin(m, fabs(Tn / 1e-4 - 1.0));
                    if (Tn < 1e-4) break;
                    T = Tn;
                }
                margin[poff + (int64_t)y * W + x] = m;
            }
        toff += (int64_t)TX * TY;
        poff += (int64_t)W * H;
    }
}

/* Per pixel (views concatenated, row-major): 1 when the walks under the two
 * projections keep the same fragments in the same order, else 0. */
int64_t same_sequences(int V, int64_t n, const int32_t* width, const int32_t* height, int tile,
                       const double* projA, const uint32_t* valsA, const uint32_t* rangesA, const double* projB,
                       const uint32_t* valsB, const uint32_t* rangesB, uint8_t* same) {
    int64_t toff = 0, poff = 0, differ = 0;
    for (int v = 0; v < V; ++v) {
        int W = width[v], H = height[v], TX = (W + tile - 1) / tile, TY = (H + tile - 1) / tile;
        int64_t vn = (int64_t)v * n;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int64_t t = toff + (int64_t)(y / tile) * TX + x / tile;
                uint32_t la = rangesA[2 * t + 1] - rangesA[2 * t], lb = rangesB[2 * t + 1] - rangesB[2 * t];
                uint32_t* A = (uint32_t*)malloc(sizeof(uint32_t) * (la + 1));
                uint32_t* Bq = (uint32_t*)malloc(sizeof(uint32_t) * (lb + 1));
                int ma = kept(projA, vn, valsA, rangesA[2 * t], rangesA[2 * t + 1], x + 0.5, y + 0.5, A);
                int mb = kept(projB, vn, valsB, rangesB[2 * t], rangesB[2 * t + 1], x + 0.5, y + 0.5, Bq);
                int eq = ma == mb && (ma == 0 || memcmp(A, Bq, sizeof(uint32_t) * (size_t)ma) == 0);
                same[poff + (int64_t)y * W + x] = (uint8_t)eq;
                differ += !eq;
                free(A);
                free(Bq);
            }
        toff += (int64_t)TX * TY;
        poff += (int64_t)W * H;
    }
    return differ;
}
