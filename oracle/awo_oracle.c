/*
 * awo_oracle.c -- CPU oracle for the avalanche-overlay hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, step-by-step CPU
 * statement of what the data-driven avalanche overlay computes (paper:
 * "Data-Driven Compute Overlays for Interactive Geographic Simulation and
 * Visualization", Sec. 3 and Sec. 5.2 "Avalanches").  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  The
 * CUDA library shares no code, header, table or constant with it.
 *
 * The paper states the method in prose only (no equations): normals from the
 * DEM, release cells chosen by a steepness range, Monte-Carlo particles per
 * release texel that move downslope with "persistence" (momentum), a
 * user-defined "random variation from the optimal path", and a "runout
 * angle" stop criterion measured between the current position and the
 * release point; the overlay colour is the maximum energy-line height
 * Z^delta_max, read as a velocity indicator (Sec. 5.2, Fig. 4 caption); a
 * mipmap of the overlay gives the level of detail (Sec. 3).  Every formula
 * below is the reading written down in the design notes of this repository;
 * each function names the passage it follows.
 *
 * Precision: one source, compiled twice.
 *   -DORC_REAL=float   FP32, the parity oracle (the paper's WebGPU storage is
 *                      FP32, and rasters are compared bit for bit);
 *   -DORC_REAL=double  FP64, used to pin closed forms and as the accuracy
 *                      reference for relaxed-precision modes.
 * It must be compiled with -ffp-contract=off and without -ffast-math so that
 * every +, -, *, / and sqrt below is one IEEE-754 correctly rounded
 * operation in ORC_REAL, in the order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_REAL
#define ORC_REAL float
#endif
typedef ORC_REAL real;

/* sqrt of a real: for FP32 the double square root rounded to float is the
 * correctly rounded float square root (double carries more than 2*24+2 bits). */
#define SQRT_RN(x) ((real)sqrt((double)(x)))

/* ------------------------------------------------------------------ */
/* Status codes (kept numerically equal to the library's so tests can  */
/* compare them; the values are part of the documented interface).     */
/* ------------------------------------------------------------------ */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EOVERFLOW = 5 };

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: */
/* As Easy as 1, 2, 3", SC'11, Sec. 4.2 / Fig. 2).  Counter-based: the  */
/* output is a bijection of the 128-bit counter under a 64-bit key.     */
/* One round: two 32x32->64 products of the even counter words with the */
/* round multipliers, then a word permutation mixing in the key; the   */
/* key is bumped by the Weyl constants between rounds.                  */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------ */
/* Parameters and statistics of one simulation (Sec. 5.2: persistence, */
/* random variation, runout angle, particles per release texel).       */
/* ------------------------------------------------------------------ */
typedef struct {
    real mu;            /* tan(runout angle)                                */
    real drag_k;        /* velocity-squared drag per metre (0 = paper)      */
    real persistence;   /* P in [0,1]                                       */
    real randomness;    /* R >= 0                                           */
    real step_scale;    /* horizontal step length in cells                  */
    real gravity;       /* m/s^2                                            */
    uint32_t traj_per_cell;
    uint32_t max_steps;
    uint64_t seed;
    int32_t release_log2; /* release texture at 2^r x the DEM resolution;   */
                          /* 0: release-list entries are DEM cells           */
} orc_params;

typedef struct {
    uint64_t total_steps; /* recorded moves, summed over trajectories      */
    uint64_t n_traj;
    uint64_t n_exited;    /* left the sampling domain                       */
    uint64_t n_capped;    /* reached max_steps                              */
    uint64_t n_stopped;   /* energy reached zero, or zero direction         */
} orc_stats;

/* ------------------------------------------------------------------ */
/* a0. Decode of quantised heights: h = q * scale, one rounding.        */
/* ------------------------------------------------------------------ */
void orc_decode_u16(const uint16_t* q, int64_t n, real scale, real* h)
{
    for (int64_t i = 0; i < n; ++i)
        h[i] = (real)q[i] * scale;
}

/* ------------------------------------------------------------------ */
/* a1. Normals and steepness (Sec. 5.1 and 5.2: "compute the surface   */
/* normals" of the stitched DEM; release selection evaluates local     */
/* steepness).  Central differences with clamped neighbours, one-sided */
/* at the border; a dimension of size 1 has zero derivative.           */
/*   gx = (h[y][xr] - h[y][xl]) / (cs * (xr - xl))                      */
/*   t2 = gx*gx + gy*gy            (tan^2 of the slope angle)           */
/*   n  = (-gx, -gy, 1) * (1 / sqrt(t2 + 1))                            */
/*   slope_deg = atan(sqrt(t2)) in degrees (display only).              */
/* nrm is SoA: nx plane, ny plane, nz plane, each W*H.                  */
/* ------------------------------------------------------------------ */
int orc_normals(const real* h, int32_t W, int32_t H, real cs,
                real* nrm, real* tan2, real* slope_deg)
{
    if (W <= 0 || H <= 0 || !(cs > 0)) return ORC_EINVAL;
    const int64_t plane = (int64_t)W * H;
    for (int32_t y = 0; y < H; ++y) {
        for (int32_t x = 0; x < W; ++x) {
            int32_t xl = x > 0 ? x - 1 : 0, xr = x < W - 1 ? x + 1 : W - 1;
            int32_t yl = y > 0 ? y - 1 : 0, yr = y < H - 1 ? y + 1 : H - 1;
            real gx = 0, gy = 0;
            if (xr > xl) {
                real den = cs * (real)(xr - xl);
                gx = (h[(int64_t)y * W + xr] - h[(int64_t)y * W + xl]) / den;
            }
            if (yr > yl) {
                real den = cs * (real)(yr - yl);
                gy = (h[(int64_t)yr * W + x] - h[(int64_t)yl * W + x]) / den;
            }
            real t2 = gx * gx + gy * gy;
            real inv = (real)1 / SQRT_RN(t2 + (real)1);
            int64_t i = (int64_t)y * W + x;
            if (nrm) {
                nrm[i] = -gx * inv;
                nrm[plane + i] = -gy * inv;
                nrm[2 * plane + i] = inv;
            }
            if (tan2) tan2[i] = t2;
            if (slope_deg)
                slope_deg[i] = (real)(atan(sqrt((double)t2)) * (180.0 / 3.14159265358979323846));
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* b. Release cells (Sec. 5.2: a texel is a potential release point if */
/* its local steepness lies in the user's range; the node outputs a    */
/* binary map).  Inclusive range on tan^2, thresholds computed in FP64 */
/* from degrees and rounded to ORC_REAL once.  Also lists the release  */
/* cell indices in increasing index order.                             */
/* ------------------------------------------------------------------ */
static real tan2_of_degrees(double deg)
{
    double t = tan(deg * (3.14159265358979323846 / 180.0));
    return (real)(t * t);
}

int orc_release(const real* tan2, int32_t W, int32_t H, double lo_deg, double hi_deg,
                uint8_t* mask, uint32_t* cells, uint32_t* n_out)
{
    if (W <= 0 || H <= 0) return ORC_EINVAL;
    if (!(lo_deg >= 0.0) || !(hi_deg < 90.0) || lo_deg > hi_deg) return ORC_EINVAL;
    real t_lo = tan2_of_degrees(lo_deg), t_hi = tan2_of_degrees(hi_deg);
    uint32_t n = 0;
    for (int64_t i = 0; i < (int64_t)W * H; ++i) {
        int sel = (t_lo <= tan2[i]) && (tan2[i] <= t_hi);
        if (mask) mask[i] = (uint8_t)sel;
        if (sel) {
            if (cells) cells[n] = (uint32_t)i;
            ++n;
        }
    }
    *n_out = n;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* b''. Release points on a texture of chosen resolution (Sec. 5.2: the */
/* user picks the texture resolution at which potential release points */
/* are evaluated).  The texture covers the DEM's extent at 2^r times    */
/* its resolution, r in [-3, 3]: Wr = W 2^r, Hr = H 2^r for r >= 0, and */
/* the ceilings of W 2^r, H 2^r for r < 0 (the last texel then reaches  */
/* past the DEM).  Texel (a, b) has its centre at                        */
/*   u = (a + 1/2) 2^-r - 1/2,  v = (b + 1/2) 2^-r - 1/2                 */
/* in cell units, clamped to the sampling domain [0, W-1] x [0, H-1]     */
/* (exact in FP32: a few fraction bits, magnitude below 2^17).  The     */
/* steepness there is the bilinear interpolation of the cells' tan^2,  */
/* with the footprint and weights of the height sampling below; a texel */
/* is a release point iff T_lo <= tan^2 <= T_hi.  At r = 0 the centres  */
/* are the cell centres, the weights are 1 and 0, and the result is     */
/* orc_release's.  Release-list entries are texel indices b Wr + a.     */
/* ------------------------------------------------------------------ */
#define ORC_RELEASE_LOG2_MAX 3

int orc_release_texture_dims(int32_t W, int32_t H, int32_t r, int64_t* Wr, int64_t* Hr)
{
    if (W <= 0 || H <= 0 || r < -ORC_RELEASE_LOG2_MAX || r > ORC_RELEASE_LOG2_MAX) return ORC_EINVAL;
    if (r >= 0) {
        *Wr = (int64_t)W << r;
        *Hr = (int64_t)H << r;
    } else {
        const int64_t q = (int64_t)1 << (-r);
        *Wr = ((int64_t)W + q - 1) / q;
        *Hr = ((int64_t)H + q - 1) / q;
    }
    if (*Wr * *Hr >= ((int64_t)1 << 31)) return ORC_EINVAL;
    return ORC_OK;
}

static real texel_axis(int64_t a, int32_t r, int32_t n)
{
    double c = ldexp((double)a + 0.5, -r) - 0.5;
    if (c < 0.0) c = 0.0;
    if (c > (double)(n - 1)) c = (double)(n - 1);
    return (real)c;
}

/* Start position of release-list entry t (a texel index of the release */
/* texture at 2^r; a cell index at r = 0).                              */
static void release_point(int32_t W, int32_t H, int32_t r, int64_t Wr, uint32_t t, real* u, real* v)
{
    *u = texel_axis((int64_t)t % Wr, r, W);
    *v = texel_axis((int64_t)t / Wr, r, H);
}

/* ------------------------------------------------------------------ */
/* Bilinear sampling of the DEM.  Positions are in cell units: cell   */
/* (x, y) has its centre at (u, v) = (x, y); the sampling domain is    */
/* u in [0, W-1], v in [0, H-1].                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t i0, i1, j0, j1;
    real fx, fy;
    real h00, h10, h01, h11; /* h[j0][i0], h[j0][i1], h[j1][i0], h[j1][i1] */
} footprint;

static footprint take_footprint(const real* h, int32_t W, int32_t H, real u, real v)
{
    footprint f;
    f.i0 = (int32_t)floor(u);
    f.j0 = (int32_t)floor(v);
    f.i1 = f.i0 + 1 < W ? f.i0 + 1 : W - 1;
    f.j1 = f.j0 + 1 < H ? f.j0 + 1 : H - 1;
    f.fx = u - (real)f.i0;
    f.fy = v - (real)f.j0;
    f.h00 = h[(int64_t)f.j0 * W + f.i0];
    f.h10 = h[(int64_t)f.j0 * W + f.i1];
    f.h01 = h[(int64_t)f.j1 * W + f.i0];
    f.h11 = h[(int64_t)f.j1 * W + f.i1];
    return f;
}

/* z = (h00 (1-fx) + h10 fx) (1-fy) + (h01 (1-fx) + h11 fx) fy */
static real bilinear_height(const footprint* f)
{
    real ox = (real)1 - f->fx, oy = (real)1 - f->fy;
    real top = f->h00 * ox + f->h10 * f->fx;
    real bot = f->h01 * ox + f->h11 * f->fx;
    return top * oy + bot * f->fy;
}

int orc_release_texture(const real* tan2, int32_t W, int32_t H, int32_t r, double lo_deg, double hi_deg,
                        uint8_t* mask, uint32_t* texels, uint32_t* n_out)
{
    int64_t Wr, Hr;
    if (orc_release_texture_dims(W, H, r, &Wr, &Hr)) return ORC_EINVAL;
    if (!(lo_deg >= 0.0) || !(hi_deg < 90.0) || lo_deg > hi_deg) return ORC_EINVAL;
    real t_lo = tan2_of_degrees(lo_deg), t_hi = tan2_of_degrees(hi_deg);
    uint32_t n = 0;
    for (int64_t t = 0; t < Wr * Hr; ++t) {
        real u, v;
        release_point(W, H, r, Wr, (uint32_t)t, &u, &v);
        footprint f = take_footprint(tan2, W, H, u, v);
        real T = bilinear_height(&f);
        int sel = (t_lo <= T) && (T <= t_hi);
        if (mask) mask[t] = (uint8_t)sel;
        if (sel) {
            if (texels) texels[n] = (uint32_t)t;
            ++n;
        }
    }
    *n_out = n;
    return ORC_OK;
}

/* Steepest-descent unit direction of the bilinear patch (Sec. 5.2:    */
/* particles follow the "optimal path" downslope).  The patch gradient */
/* in height per cell is (a, b):                                       */
/*   a = (h10-h00)(1-fy) + (h11-h01) fy,  b = (h01-h00)(1-fx) + (h11-h10) fx */
/* Its direction does not depend on the cell size.  g = -(a,b)/|(a,b)|,*/
/* normalised by one reciprocal of the rounded norm.  A zero gradient  */
/* returns the fallback direction.                                     */
static void downslope(const footprint* f, real fb_x, real fb_y, real* gx, real* gy)
{
    real ox = (real)1 - f->fx, oy = (real)1 - f->fy;
    real a = (f->h10 - f->h00) * oy + (f->h11 - f->h01) * f->fy;
    real b = (f->h01 - f->h00) * ox + (f->h11 - f->h10) * f->fx;
    real n2 = a * a + b * b;
    if (n2 == (real)0) {
        *gx = fb_x;
        *gy = fb_y;
        return;
    }
    real inv = (real)1 / SQRT_RN(n2);
    *gx = -a * inv;
    *gy = -b * inv;
}

/* Cell containing a position: floor(u + 1/2) per axis, evaluated      */
/* exactly as floor(u) + [u - floor(u) >= 1/2] (no rounding of u+1/2). */
static int64_t cell_of(int32_t W, real u, real v)
{
    int64_t i0 = (int64_t)floor(u), j0 = (int64_t)floor(v);
    int64_t cx = i0 + ((u - (real)i0) >= (real)0.5 ? 1 : 0);
    int64_t cy = j0 + ((v - (real)j0) >= (real)0.5 ? 1 : 0);
    return cy * W + cx;
}

/* Uniform variate in [-1, 1) from the top 24 bits of a Philox word,   */
/* exact in FP32: (w >> 8) * 2^-23 - 1.                                */
static real uniform_pm1(uint32_t w)
{
    return (real)(w >> 8) * (real)(1.0 / 8388608.0) - (real)1;
}

/* Random words of move n of trajectory (cell, j): Philox block         */
/* ctr = (cell, j, n >> 1, 0), key = (seed lo, seed hi); even moves take */
/* words 0 and 1, odd moves words 2 and 3.                              */
static void draw_pair(uint32_t cell, uint32_t j, uint32_t n, uint64_t seed, uint32_t* wx, uint32_t* wy)
{
    uint32_t ctr[4] = {cell, j, n >> 1, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    if ((n & 1u) == 0u) {
        *wx = r[0];
        *wy = r[1];
    } else {
        *wx = r[2];
        *wy = r[3];
    }
}

/* The two uniforms of move n of trajectory (cell, j), for tests.      */
void orc_draw(uint32_t cell, uint32_t j, uint32_t n, uint64_t seed, real xi[2])
{
    uint32_t wx, wy;
    draw_pair(cell, j, n, seed, &wx, &wy);
    xi[0] = uniform_pm1(wx);
    xi[1] = uniform_pm1(wy);
}

/* ------------------------------------------------------------------ */
/* c. One trajectory (Sec. 5.2, "avalanche trajectory node").         */
/* State: position p = (u, v) in cells, unit direction d, energy-line  */
/* height e in metres (kinetic energy per unit weight, v^2 / 2g), and  */
/* the sampled height z at p.                                           */
/*   start: p0 = release cell centre (or release texel centre), e0 = 0, */
/*          d0 = g(p0) (zero if flat); the start is a visit of the cell  */
/*          of p0 with e = 0.  The random stream is keyed by the list    */
/*          entry (cell or texel index).                                 */
/*   move n = 0, 1, ... while n < max_steps:                            */
/*     g  = steepest-descent direction at p_n (fallback d_n)            */
/*     xi = two uniforms in [-1,1) from Philox (cell, j, n)             */
/*     r  = (P d_n + (1-P) g) + R xi ; stop if r = 0                     */
/*     d  = r / |r| ; p' = p + s d (s = step length in cells)           */
/*     leave the domain -> exit (not recorded)                          */
/*     e' = (e - (k D) e) + (z - z') - mu D     (D = s * cs metres)     */
/*     e' <= 0 -> stop at p (not recorded): the runout-angle criterion  */
/*       with k = 0 is exactly e_n = z0 - z_n - mu * (path length)      */
/*     else move, record a visit of cell(p') with e'                    */
/*   reaching max_steps moves -> capped.                                */
/* visit(cell, e): count += 1; maxe = max(maxe, e).                     */
/* The per-step trace (optional) receives the state after each move.  */
/* ------------------------------------------------------------------ */
enum { END_CAPPED = 0, END_EXITED = 1, END_STOPPED = 2 };

typedef struct {
    int64_t cap;     /* capacity of the arrays below */
    int64_t n;       /* entries written (moves recorded, plus the start) */
    real* u;
    real* v;
    real* e;
    int64_t* cell;
    int32_t end;     /* END_* */
} orc_trace_buf;

static int run_trajectory(const real* h, int32_t W, int32_t H, real cs, uint32_t cell, real u0, real v0,
                          uint32_t j, const orc_params* p, uint64_t* count, real* maxe, orc_stats* st,
                          orc_trace_buf* tr)
{
    const real P = p->persistence, R = p->randomness, s = p->step_scale;
    const real oneP = (real)1 - P;
    const real D = s * cs;
    const real kD = p->drag_k * D, muD = p->mu * D;

    real u = u0, v = v0;
    footprint f = take_footprint(h, W, H, u, v);
    real z = bilinear_height(&f);
    real e = 0;
    real dx, dy;
    downslope(&f, (real)0, (real)0, &dx, &dy);

    /* the start is a visit of the release cell */
    if (count) {
        int64_t c = cell_of(W, u, v);
        count[c] += 1;
        if (e > maxe[c]) maxe[c] = e;
    }
    if (tr && tr->n < tr->cap) {
        tr->u[tr->n] = u; tr->v[tr->n] = v; tr->e[tr->n] = e; tr->cell[tr->n] = cell_of(W, u, v);
        tr->n++;
    }

    int end = END_CAPPED;
    uint32_t n = 0;
    while (n < p->max_steps) {
        real gx, gy;
        f = take_footprint(h, W, H, u, v);
        downslope(&f, dx, dy, &gx, &gy);

        uint32_t wx, wy;
        draw_pair(cell, j, n, p->seed, &wx, &wy);
        real xix = uniform_pm1(wx), xiy = uniform_pm1(wy);

        real rx = (P * dx + oneP * gx) + R * xix;
        real ry = (P * dy + oneP * gy) + R * xiy;
        real r2 = rx * rx + ry * ry;
        if (r2 == (real)0) { end = END_STOPPED; break; }
        real inv = (real)1 / SQRT_RN(r2);
        dx = rx * inv;
        dy = ry * inv;

        real u1 = u + s * dx, v1 = v + s * dy;
        if (!(u1 >= (real)0 && u1 <= (real)(W - 1) && v1 >= (real)0 && v1 <= (real)(H - 1))) {
            end = END_EXITED;
            break;
        }
        footprint f1 = take_footprint(h, W, H, u1, v1);
        real z1 = bilinear_height(&f1);
        real e1 = (e - kD * e) + (z - z1) - muD;
        if (!(e1 > (real)0)) { end = END_STOPPED; break; }

        u = u1; v = v1; z = z1; e = e1;
        ++n;
        int64_t c = cell_of(W, u, v);
        if (count) {
            count[c] += 1;
            if (e > maxe[c]) maxe[c] = e;
        }
        if (st) st->total_steps++;
        if (tr && tr->n < tr->cap) {
            tr->u[tr->n] = u; tr->v[tr->n] = v; tr->e[tr->n] = e; tr->cell[tr->n] = c;
            tr->n++;
        }
    }
    if (st) {
        st->n_traj++;
        if (end == END_CAPPED) st->n_capped++;
        else if (end == END_EXITED) st->n_exited++;
        else st->n_stopped++;
    }
    if (tr) tr->end = end;
    return end;
}

static int check_params(int32_t W, int32_t H, real cs, const orc_params* p)
{
    if (W <= 0 || H <= 0 || !(cs > 0) || !p) return ORC_EINVAL;
    if (!(p->persistence >= 0 && p->persistence <= 1)) return ORC_EINVAL;
    if (!(p->randomness >= 0) || !(p->mu >= 0) || !(p->drag_k >= 0)) return ORC_EINVAL;
    if (!(p->step_scale > 0) || !(p->step_scale <= 1)) return ORC_EINVAL;
    if (!(p->gravity > 0)) return ORC_EINVAL;
    if (!(p->drag_k * (p->step_scale * cs) < (real)1)) return ORC_EINVAL;
    int64_t Wr, Hr;
    if (orc_release_texture_dims(W, H, p->release_log2, &Wr, &Hr)) return ORC_EINVAL;
    return ORC_OK;
}


/* Runs traj_per_cell trajectories from every listed release cell (or   */
/* texel, when p->release_log2 != 0) and accumulates visits into count  */
/* (uint64, caller zero-fills) and maxe (caller zero-fills).  Stats are  */
/* accumulated into *st.                                                */
int orc_simulate(const real* h, int32_t W, int32_t H, real cs, const uint32_t* cells, uint32_t n_cells,
                 const orc_params* p, uint64_t* count, real* maxe, orc_stats* st)
{
    int rc = check_params(W, H, cs, p);
    if (rc) return rc;
    int64_t Wr, Hr;
    orc_release_texture_dims(W, H, p->release_log2, &Wr, &Hr);
    const int64_t n_entries = Wr * Hr;
    for (uint32_t c = 0; c < n_cells; ++c) {
        if ((int64_t)cells[c] >= n_entries) return ORC_EINVAL;
        real u0, v0;
        release_point(W, H, p->release_log2, Wr, cells[c], &u0, &v0);
        for (uint32_t j = 0; j < p->traj_per_cell; ++j)
            run_trajectory(h, W, H, cs, cells[c], u0, v0, j, p, count, maxe, st, NULL);
    }
    return ORC_OK;
}

/* One trajectory with its full trace (start + every recorded move).   */
int orc_trace(const real* h, int32_t W, int32_t H, real cs, uint32_t cell, uint32_t j,
              const orc_params* p, int64_t cap, real* u, real* v, real* e, int64_t* cells,
              int64_t* n_out, int32_t* end_out)
{
    int rc = check_params(W, H, cs, p);
    if (rc) return rc;
    int64_t Wr, Hr;
    orc_release_texture_dims(W, H, p->release_log2, &Wr, &Hr);
    if ((int64_t)cell >= Wr * Hr) return ORC_EINVAL;
    real u0, v0;
    release_point(W, H, p->release_log2, Wr, cell, &u0, &v0);
    orc_trace_buf tr = {cap, 0, u, v, e, cells, 0};
    run_trajectory(h, W, H, cs, cell, u0, v0, j, p, NULL, NULL, NULL, &tr);
    *n_out = tr.n;
    *end_out = tr.end;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Soft-deposit mode (differentiable extension; the paper has no        */
/* gradients).  The path is the same as in the hard mode (same FP32     */
/* arithmetic in the FP32 build) but the energy no longer stops the     */
/* particle: each particle carries a survival S (S_0 = 1) that decays   */
/* by the logistic function of its energy-line height,                  */
/*   S_n = S_{n-1} * sigma(e_n / tau),  sigma(x) = 1 / (1 + exp(-x)),     */
/* and deposits the mass it loses, w (S_{n-1} - S_n), at the cell of     */
/* p_n.  The particle ends when it leaves the domain, reaches max_steps, */
/* has no direction, or S_n < 1e-7; the remainder w S_last goes to the   */
/* last cell reached, so a particle deposits exactly w.  Energy,         */
/* survival and deposits are evaluated in FP64 here.                     */
/* ------------------------------------------------------------------ */
#define SOFT_S_MIN 1e-7

typedef struct {
    int64_t n;         /* moves made */
    int64_t cap;       /* capacity of the arrays */
    double* e;         /* e_1 .. e_n */
    double* S;         /* S_1 .. S_n */
    int64_t* cell;     /* cell of p_0 .. p_n (n + 1 entries) */
} soft_path;

/* One soft particle: fills path (when non-null) and returns the number
 * of moves.  The direction and positions follow run_trajectory exactly. */
static int64_t soft_particle(const real* h, int32_t W, int32_t H, real cs, uint32_t cell, uint32_t j,
                             const orc_params* p, double tau, soft_path* sp)
{
    const real P = p->persistence, R = p->randomness, s = p->step_scale;
    const real oneP = (real)1 - P;
    const real D = s * cs;
    const double kD = (double)p->drag_k * (double)D, muD = (double)p->mu * (double)D;

    real u = (real)(cell % (uint32_t)W), v = (real)(cell / (uint32_t)W);
    footprint f = take_footprint(h, W, H, u, v);
    double z = (double)bilinear_height(&f);
    double e = 0.0, S = 1.0;
    real dx, dy;
    downslope(&f, (real)0, (real)0, &dx, &dy);
    if (sp) sp->cell[0] = cell_of(W, u, v);
    int64_t n = 0;
    while ((uint32_t)n < p->max_steps) {
        real gx, gy;
        f = take_footprint(h, W, H, u, v);
        downslope(&f, dx, dy, &gx, &gy);
        uint32_t wx, wy;
        draw_pair(cell, j, (uint32_t)n, p->seed, &wx, &wy);
        real xix = uniform_pm1(wx), xiy = uniform_pm1(wy);
        real rx = (P * dx + oneP * gx) + R * xix;
        real ry = (P * dy + oneP * gy) + R * xiy;
        real r2 = rx * rx + ry * ry;
        if (r2 == (real)0) break;
        real inv = (real)1 / SQRT_RN(r2);
        dx = rx * inv;
        dy = ry * inv;
        real u1 = u + s * dx, v1 = v + s * dy;
        if (!(u1 >= (real)0 && u1 <= (real)(W - 1) && v1 >= (real)0 && v1 <= (real)(H - 1))) break;
        footprint f1 = take_footprint(h, W, H, u1, v1);
        double z1 = (double)bilinear_height(&f1);
        double e1 = (e - kD * e) + (z - z1) - muD;
        double S1 = S / (1.0 + exp(-e1 / tau));
        u = u1; v = v1; z = z1; e = e1; S = S1;
        ++n;
        if (sp) {
            if (n >= sp->cap) return -1;
            sp->e[n] = e;
            sp->S[n] = S;
            sp->cell[n] = cell_of(W, u, v);
        }
        if (S < SOFT_S_MIN) break;
    }
    if (sp) sp->n = n;
    return n;
}

static int soft_path_alloc(soft_path* sp, uint32_t max_steps)
{
    sp->cap = (int64_t)max_steps + 2;
    sp->e = (double*)malloc(sizeof(double) * sp->cap);
    sp->S = (double*)malloc(sizeof(double) * sp->cap);
    sp->cell = (int64_t*)malloc(sizeof(int64_t) * sp->cap);
    if (!sp->e || !sp->S || !sp->cell) {
        free(sp->e); free(sp->S); free(sp->cell);
        return ORC_ENOMEM;
    }
    sp->e[0] = 0.0;
    sp->S[0] = 1.0;
    return ORC_OK;
}

static void soft_path_free(soft_path* sp) { free(sp->e); free(sp->S); free(sp->cell); }

/* Soft deposits of every particle of every listed release cell, weight
 * weight[c] per particle of entry c, accumulated into deposit (FP64, W*H). */
int orc_soft_forward(const real* h, int32_t W, int32_t H, real cs, const uint32_t* cells, uint32_t n_cells,
                     const double* weight, const orc_params* p, double tau, double* deposit, orc_stats* st)
{
    int rc = check_params(W, H, cs, p);
    if (rc) return rc;
    if (!(tau > 0) || p->release_log2 != 0) return ORC_EINVAL; /* soft mode: DEM cells only */
    soft_path sp;
    if (soft_path_alloc(&sp, p->max_steps)) return ORC_ENOMEM;
    for (uint32_t c = 0; c < n_cells; ++c) {
        if ((int64_t)cells[c] >= (int64_t)W * H) { soft_path_free(&sp); return ORC_EINVAL; }
        for (uint32_t j = 0; j < p->traj_per_cell; ++j) {
            soft_particle(h, W, H, cs, cells[c], j, p, tau, &sp);
            double w = weight[c];
            for (int64_t m = 1; m <= sp.n; ++m) deposit[sp.cell[m]] += w * (sp.S[m - 1] - sp.S[m]);
            deposit[sp.cell[sp.n]] += w * sp.S[sp.n];
            if (st) { st->n_traj++; st->total_steps += (uint64_t)sp.n; }
        }
    }
    soft_path_free(&sp);
    return ORC_OK;
}

/* Reverse-mode gradient (FP64) of L = sum_cells G_c D_c-linearised loss:
 * given G = dL/dD (W*H), returns dL/dlog(mu), dL/dlog(k) in grad_theta[0..1]
 * (accumulated) and dL/dw per release-list entry (accumulated).  Per
 * particle, the deposit functional J = w [sum_m G(c_m)(S_{m-1} - S_m) +
 * G(c_n) S_n] is differentiated by the adjoint sweep
 *   a_m     = dJ/dS_m (direct) = w (G(c_{m+1}) - G(c_m))  (m < n),  0 (m = n:
 *             the last move's deposit plus the remainder is w S_{n-1})
 *   abar_m  = a_m + sigma_{m+1} abar_{m+1}     (S_{m+1} = S_m sigma_{m+1})
 *   lam_m   = dJ/de_m = abar_m S_{m-1} sigma'(e_m) + (1 - k D) lam_{m+1},
 *             sigma'(e) = sigma (1 - sigma) / tau
 *   dJ/dmu  = -D sum_m lam_m,   dJ/dk = -D sum_m lam_m e_{m-1}
 * over the stored path (the path itself does not depend on mu, k, w). */
int orc_soft_gradient(const real* h, int32_t W, int32_t H, real cs, const uint32_t* cells, uint32_t n_cells,
                      const double* weight, const orc_params* p, double tau, const double* G,
                      double* grad_theta, double* grad_weight, double* grad_theta_abs)
{
    int rc = check_params(W, H, cs, p);
    if (rc) return rc;
    if (!(tau > 0) || p->release_log2 != 0) return ORC_EINVAL; /* soft mode: DEM cells only */
    soft_path sp;
    if (soft_path_alloc(&sp, p->max_steps)) return ORC_ENOMEM;
    const double D = (double)(p->step_scale * cs);
    const double kD = (double)p->drag_k * D;
    double* abar = (double*)malloc(sizeof(double) * sp.cap);
    if (!abar) { soft_path_free(&sp); return ORC_ENOMEM; }
    for (uint32_t c = 0; c < n_cells; ++c) {
        if ((int64_t)cells[c] >= (int64_t)W * H) { free(abar); soft_path_free(&sp); return ORC_EINVAL; }
        const double w = weight[c];
        for (uint32_t j = 0; j < p->traj_per_cell; ++j) {
            soft_particle(h, W, H, cs, cells[c], j, p, tau, &sp);
            const int64_t n = sp.n;
            /* dJ/dw */
            double jw = 0.0;
            for (int64_t m = 1; m <= n; ++m) jw += G[sp.cell[m]] * (sp.S[m - 1] - sp.S[m]);
            jw += G[sp.cell[n]] * sp.S[n];
            grad_weight[c] += jw;
            /* adjoint of S_m, backwards: J depends on S_m directly through
             * w (G(c_{m+1}) - G(c_m)) (or w G(c_n) at the end) and through
             * S_{m+1} = S_m sigma_{m+1} */
            for (int64_t m = n; m >= 1; --m) {
                double direct = (m < n) ? w * (G[sp.cell[m + 1]] - G[sp.cell[m]]) : 0.0;
                double sig_next = (m < n) ? sp.S[m + 1] / sp.S[m] : 0.0;
                abar[m] = direct + ((m < n) ? sig_next * abar[m + 1] : 0.0);
            }
            /* adjoint of e_m: S_m = S_{m-1} sigma(e_m / tau) and e_{m+1} = e_m (1 - kD) + ... */
            double lam_next = 0.0, dmu = 0.0, dk = 0.0;
            for (int64_t m = n; m >= 1; --m) {
                double sig = sp.S[m] / sp.S[m - 1];
                double dsig = sig * (1.0 - sig) / tau;
                double lam = abar[m] * sp.S[m - 1] * dsig + (1.0 - kD) * lam_next;
                dmu += -D * lam;
                dk += -D * lam * sp.e[m - 1];
                lam_next = lam;
            }
            grad_theta[0] += (double)p->mu * dmu;   /* d/dlog(mu) = mu d/dmu */
            grad_theta[1] += (double)p->drag_k * dk;
            if (grad_theta_abs) { /* sum of |per-particle terms|: the conditioning of the sum over particles */
                grad_theta_abs[0] += fabs((double)p->mu * dmu);
                grad_theta_abs[1] += fabs((double)p->drag_k * dk);
            }
        }
    }
    free(abar);
    soft_path_free(&sp);
    return ORC_OK;
}

/* c'. Velocity indicator per cell from the maximum energy-line height  */
/* (Fig. 4 caption: the colour encodes Z^delta_max, read as velocity):  */
/* vel = sqrt((2 g) * maxe).                                            */
void orc_finalize(const real* maxe, int64_t n, real gravity, real* vel)
{
    real g2 = (real)2 * gravity;
    for (int64_t i = 0; i < n; ++i)
        vel[i] = SQRT_RN(g2 * maxe[i]);
}

/* ------------------------------------------------------------------ */
/* d. Level of detail (Sec. 3: "from the high-resolution overlay       */
/* texture, we then compute a mipmap").  Level l+1 from level l by     */
/* 2x2 blocks, size ceil(W_l / 2) x ceil(H_l / 2); a block that hangs  */
/* over the edge uses the texels present.  Counts: sum of the block,   */
/* saturated to 2^32-1; velocity: max of the block.  count_lv[l-1] and */
/* vel_lv[l-1] receive level l, for l = 1 .. levels-1.                 */
/* ------------------------------------------------------------------ */
int orc_lod(const uint32_t* count, const real* vel, int32_t W, int32_t H, int32_t levels,
            uint32_t* const* count_lv, real* const* vel_lv)
{
    if (W <= 0 || H <= 0 || levels < 1 || levels > 16) return ORC_EINVAL;
    const uint32_t* pc = count;
    const real* pv = vel;
    int32_t w = W, hgt = H;
    for (int32_t l = 1; l < levels; ++l) {
        int32_t w2 = (w + 1) / 2, h2 = (hgt + 1) / 2;
        uint32_t* oc = count_lv[l - 1];
        real* ov = vel_lv[l - 1];
        for (int32_t y = 0; y < h2; ++y) {
            for (int32_t x = 0; x < w2; ++x) {
                uint64_t sum = 0;
                real m = 0;
                int first = 1;
                for (int32_t dy = 0; dy < 2; ++dy) {
                    for (int32_t dx = 0; dx < 2; ++dx) {
                        int32_t sx = 2 * x + dx, sy = 2 * y + dy;
                        if (sx >= w || sy >= hgt) continue;
                        int64_t si = (int64_t)sy * w + sx;
                        sum += pc[si];
                        if (first || pv[si] > m) m = pv[si];
                        first = 0;
                    }
                }
                oc[(int64_t)y * w2 + x] = sum > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)sum;
                ov[(int64_t)y * w2 + x] = m;
            }
        }
        pc = oc;
        pv = ov;
        w = w2;
        hgt = h2;
    }
    return ORC_OK;
}

/* Size of the real type this build computes in (4 or 8). */
int orc_real_size(void) { return (int)sizeof(real); }

/* ------------------------------------------------------------------ */
/* Compose pass (Sec. 3: the overlay is alpha-blended over the base map; */
/* Fig. 4: colour encodes Z^delta_max, read as velocity).  Per texel:    */
/*   k: the ramp segment with value[k] <= x <= value[k+1] (x clamped to   */
/*      the first and last stops),  t = (x - value[k]) / (value[k+1] -    */
/*      value[k]),  c = rgb[k] + t (rgb[k+1] - rgb[k])  per channel;      */
/*   a = alpha when count >= count_min, else 0;                          */
/*   with a base: out.rgb = rint(a c + (1 - a) base.rgb), out.a = base.a; */
/*   without:     out.rgb = rint(c), out.a = rint(255 a).                 */
/* FP32 in the FP32 build, round half to even.                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t n_stops;
    float value[16];
    uint8_t rgb[16][3];
    uint8_t pad[4];
    float alpha;
    uint32_t count_min;
} orc_colormap;

static uint8_t to_u8(real x)
{
    if (!(x > (real)0)) return 0;
    if (x > (real)255) return 255;
    return (uint8_t)rint((double)x);
}

int orc_compose(const real* value, const uint32_t* count, int64_t n, const orc_colormap* cm, const uint8_t* base,
                uint8_t* out)
{
    if (!cm || cm->n_stops < 2 || cm->n_stops > 16) return ORC_EINVAL;
    for (int k = 0; k + 1 < cm->n_stops; ++k)
        if (!(cm->value[k] < cm->value[k + 1])) return ORC_EINVAL;
    const real alpha = (real)cm->alpha;
    for (int64_t i = 0; i < n; ++i) {
        real x = value[i];
        const int last = cm->n_stops - 1;
        if (!(x > (real)cm->value[0])) x = (real)cm->value[0];
        if (x > (real)cm->value[last]) x = (real)cm->value[last];
        int k = 0;
        while (k + 1 < last && x >= (real)cm->value[k + 1]) ++k;
        const real t = (x - (real)cm->value[k]) / ((real)cm->value[k + 1] - (real)cm->value[k]);
        const real a = count[i] >= cm->count_min ? alpha : (real)0;
        for (int ch = 0; ch < 3; ++ch) {
            const real c0 = (real)cm->rgb[k][ch], c1 = (real)cm->rgb[k + 1][ch];
            const real c = c0 + t * (c1 - c0);
            if (base)
                out[4 * i + ch] = to_u8(a * c + ((real)1 - a) * (real)base[4 * i + ch]);
            else
                out[4 * i + ch] = to_u8(c);
        }
        out[4 * i + 3] = base ? base[4 * i + 3] : to_u8((real)255 * a);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Snow cover (Sec. 5.1: the user sets the snow-line altitude, the      */
/* maximum steepness and blending factors; snow-covered texels are      */
/* white with alpha the blending factor).  Per texel with height h and  */
/* normal z-component nz (nz = cos of the slope angle):                 */
/*   a_alt   = smoothstep(L - b/2, L + b/2, h)                           */
/*   a_slope = smoothstep(cos(m + c/2), cos(m - c/2), nz)                */
/*   alpha   = a_alt * a_slope                                           */
/* smoothstep(e0, e1, x) = t t (3 - 2 t), t = clamp((x - e0)/(e1 - e0)), */
/* a step (x >= e0) when e0 == e1.  The four edges are computed in FP64  */
/* from the parameters and rounded to FP32 once.                         */
/* ------------------------------------------------------------------ */
static real smooth_step(real e0, real e1, real x)
{
    if (e1 == e0) return x >= e0 ? (real)1 : (real)0;
    real t = (x - e0) / (e1 - e0);
    if (t < (real)0) t = 0;
    if (t > (real)1) t = 1;
    return t * t * ((real)3 - (real)2 * t);
}

int orc_snow_cover(const real* h, const real* nz, int64_t n, double snow_line, double blend_alt, double max_slope_deg,
                   double blend_slope_deg, real* alpha, uint8_t* rgba)
{
    if (!(blend_alt >= 0) || !(blend_slope_deg >= 0) || !(max_slope_deg >= 0) || !(max_slope_deg <= 90))
        return ORC_EINVAL;
    const double r = 3.14159265358979323846 / 180.0;
    const real a0 = (real)(snow_line - 0.5 * blend_alt), a1 = (real)(snow_line + 0.5 * blend_alt);
    double s_lo = max_slope_deg + 0.5 * blend_slope_deg, s_hi = max_slope_deg - 0.5 * blend_slope_deg;
    if (s_lo > 90.0) s_lo = 90.0;
    if (s_hi < 0.0) s_hi = 0.0;
    const real c0 = (real)cos(s_lo * r), c1 = (real)cos(s_hi * r);
    for (int64_t i = 0; i < n; ++i) {
        real a = smooth_step(a0, a1, h[i]) * smooth_step(c0, c1, nz[i]);
        alpha[i] = a;
        if (rgba) {
            rgba[4 * i + 0] = rgba[4 * i + 1] = rgba[4 * i + 2] = 255;
            rgba[4 * i + 3] = to_u8((real)255 * a);
        }
    }
    return ORC_OK;
}
