/*
 * Seeded synthetic problem generators: system matrices of the three
 * workload families (parallel-beam CT, straight-ray seismic traveltime,
 * pencil-beam radiotherapy dose influence).
 *
 * This file builds INPUTS only.  It holds none of the projection or
 * superiorization arithmetic; both the FP64 oracle and the CUDA path consume
 * what it produces.  Every matrix is emitted as CSR in two passes: a count
 * pass that fills per-row lengths, and a fill pass that writes column indices
 * (strictly increasing within a row) and FP32 values at caller-provided row
 * offsets.  Rows are independent, so both passes are row-parallel (OpenMP)
 * and deterministic.
 *
 * Ray tracing follows Siddon's method (R. L. Siddon, "Fast calculation of the
 * exact radiological path for a three-dimensional CT array", Med. Phys. 12,
 * 1985): the parametric values at which a segment crosses the vertical and the
 * horizontal grid lines are merged in increasing order; each consecutive pair
 * bounds one cell, identified from the pair's midpoint, and the pair's
 * parametric difference times the segment length is the intersection length.
 *
 * Build with -ffp-contract=off so x86-64 and aarch64 produce the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* A 2-D grid of nx columns by ny rows; cell (iy, ix) has index iy*nx+ix and
 * covers [ox+ix*hx, ox+(ix+1)*hx] x [oy+iy*hy, oy+(iy+1)*hy]. */
typedef struct {
    int nx, ny;
    double ox, oy, hx, hy;
} grid2d;

/* Clip the line p0 + t*d (t real) to the grid box.  Returns 0 when the line
 * misses the box or only touches it. */
static int clip_line(const grid2d* g, double p0x, double p0y, double dx, double dy,
                     double tlo, double thi, double* t0, double* t1) {
    double lo = tlo, hi = thi;
    const double bx0 = g->ox, bx1 = g->ox + g->nx * g->hx;
    const double by0 = g->oy, by1 = g->oy + g->ny * g->hy;
    if (dx != 0.0) {
        double a = (bx0 - p0x) / dx, b = (bx1 - p0x) / dx;
        if (a > b) { double s = a; a = b; b = s; }
        if (a > lo) lo = a;
        if (b < hi) hi = b;
    } else if (p0x <= bx0 || p0x >= bx1) {
        return 0;
    }
    if (dy != 0.0) {
        double a = (by0 - p0y) / dy, b = (by1 - p0y) / dy;
        if (a > b) { double s = a; a = b; b = s; }
        if (a > lo) lo = a;
        if (b < hi) hi = b;
    } else if (p0y <= by0 || p0y >= by1) {
        return 0;
    }
    if (!(hi > lo)) return 0;
    *t0 = lo;
    *t1 = hi;
    return 1;
}

/* Trace the part of the segment p0 + t*d, t in [tlo, thi], that lies in the
 * grid; |d| = 1 so t is arc length.  Writes at most cap (cell, length) pairs
 * sorted by cell index and returns the number of cells crossed. */
static int trace(const grid2d* g, double p0x, double p0y, double dx, double dy,
                 double tlo, double thi, int32_t* cells, float* lens, int cap) {
    double t0, t1;
    if (!clip_line(g, p0x, p0y, dx, dy, tlo, thi, &t0, &t1)) return 0;
    const double minseg = 1e-9 * (g->hx < g->hy ? g->hx : g->hy);

    /* crossing parameters of the vertical lines x = ox + k*hx inside (t0, t1) */
    int kx = 0, kxend = 0, kxstep = 0;
    if (dx != 0.0) {
        double xa = p0x + t0 * dx, xb = p0x + t1 * dx;
        double xmin = xa < xb ? xa : xb, xmax = xa < xb ? xb : xa;
        int kmin = (int)ceil((xmin - g->ox) / g->hx);
        int kmax = (int)floor((xmax - g->ox) / g->hx);
        if (kmin < 0) kmin = 0;
        if (kmax > g->nx) kmax = g->nx;
        if (dx > 0) { kx = kmin; kxend = kmax + 1; kxstep = 1; }
        else { kx = kmax; kxend = kmin - 1; kxstep = -1; }
    }
    int ky = 0, kyend = 0, kystep = 0;
    if (dy != 0.0) {
        double ya = p0y + t0 * dy, yb = p0y + t1 * dy;
        double ymin = ya < yb ? ya : yb, ymax = ya < yb ? yb : ya;
        int kmin = (int)ceil((ymin - g->oy) / g->hy);
        int kmax = (int)floor((ymax - g->oy) / g->hy);
        if (kmin < 0) kmin = 0;
        if (kmax > g->ny) kmax = g->ny;
        if (dy > 0) { ky = kmin; kyend = kmax + 1; kystep = 1; }
        else { ky = kmax; kyend = kmin - 1; kystep = -1; }
    }

    int cnt = 0;
    double tprev = t0;
    for (;;) {
        double tx = INFINITY, ty = INFINITY;
        if (kxstep != 0 && kx != kxend) {
            tx = (g->ox + kx * g->hx - p0x) / dx;
            if (tx <= tprev) { kx += kxstep; continue; }
        }
        if (kystep != 0 && ky != kyend) {
            ty = (g->oy + ky * g->hy - p0y) / dy;
            if (ty <= tprev) { ky += kystep; continue; }
        }
        double tnext = tx < ty ? tx : ty;
        if (tnext > t1) tnext = t1;
        if (tnext - tprev > minseg) {
            double tm = 0.5 * (tprev + tnext);
            int ix = (int)floor((p0x + tm * dx - g->ox) / g->hx);
            int iy = (int)floor((p0y + tm * dy - g->oy) / g->hy);
            if (ix < 0) ix = 0;
            if (ix >= g->nx) ix = g->nx - 1;
            if (iy < 0) iy = 0;
            if (iy >= g->ny) iy = g->ny - 1;
            if (cells && cnt < cap) {
                cells[cnt] = iy * g->nx + ix;
                lens[cnt] = (float)(tnext - tprev);
            }
            cnt++;
        }
        if (tnext >= t1) break;
        tprev = tnext;
        if (tx <= ty) kx += kxstep;
        if (ty <= tx) ky += kystep;
    }
    if (cells && cnt <= cap) {
        /* The traversal is monotone in iy (direction sign(dy)) and in ix
         * (sign(dx)).  Sort by index = (iy, ix) in O(cnt): reverse the whole
         * run when iy decreases, then reverse each equal-iy run whose ix
         * decreases. */
        if (dy < 0) {
            for (int a = 0, b = cnt - 1; a < b; ++a, --b) {
                int32_t c = cells[a]; cells[a] = cells[b]; cells[b] = c;
                float l = lens[a]; lens[a] = lens[b]; lens[b] = l;
            }
        }
        double ixdir = (dy < 0) ? -dx : dx;
        if (ixdir < 0) {
            int a = 0;
            while (a < cnt) {
                int row = cells[a] / g->nx, e = a;
                while (e + 1 < cnt && cells[e + 1] / g->nx == row) ++e;
                for (int p = a, q = e; p < q; ++p, --q) {
                    int32_t c = cells[p]; cells[p] = cells[q]; cells[q] = c;
                    float l = lens[p]; lens[p] = lens[q]; lens[q] = l;
                }
                a = e + 1;
            }
        }
    }
    return cnt;
}

/* ---------------------------------------------------------------- CT ---- */
/* Parallel-beam CT on an N x N image covering [-1,1]^2 (pixel size 2/N).
 * Row r = a*nbin + k is the ray at angle theta_a = a*pi/nang with detector
 * offset s_k = (k - (nbin-1)/2) * (2*sqrt(2)/nbin): points s*n + t*u with
 * u = (cos, sin), n = (-sin, cos).  Image row i spans y in [-1+i*h, -1+(i+1)*h],
 * column j spans x likewise; pixel index i*N + j. */
static void ct_ray(int N, int nang, int nbin, int r, grid2d* g, double* px, double* py,
                   double* dx, double* dy) {
    g->nx = N; g->ny = N; g->ox = -1.0; g->oy = -1.0; g->hx = 2.0 / N; g->hy = 2.0 / N;
    int a = r / nbin, k = r % nbin;
    double th = M_PI * (double)a / (double)nang;
    double s = ((double)k - 0.5 * (nbin - 1)) * (2.0 * sqrt(2.0) / (double)nbin);
    double c = cos(th), sn = sin(th);
    *dx = c; *dy = sn;
    *px = -s * sn; *py = s * c;
}

int64_t synth_ct_count(int N, int nang, int nbin, int32_t* row_len) {
    int64_t m = (int64_t)nang * nbin, tot = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : tot)
    for (int64_t r = 0; r < m; ++r) {
        grid2d g; double px, py, dx, dy;
        ct_ray(N, nang, nbin, (int)r, &g, &px, &py, &dx, &dy);
        int c = trace(&g, px, py, dx, dy, -1e30, 1e30, NULL, NULL, 0);
        row_len[r] = c;
        tot += c;
    }
    return tot;
}

void synth_ct_fill(int N, int nang, int nbin, const int64_t* row_ptr, int32_t* col, float* val) {
    int64_t m = (int64_t)nang * nbin;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < m; ++r) {
        grid2d g; double px, py, dx, dy;
        ct_ray(N, nang, nbin, (int)r, &g, &px, &py, &dx, &dy);
        int cap = (int)(row_ptr[r + 1] - row_ptr[r]);
        trace(&g, px, py, dx, dy, -1e30, 1e30, col + row_ptr[r], val + row_ptr[r], cap);
    }
}

/* Chord length of CT ray r through the image square (closed form of the
 * slab clip), used to check the tracer. */
double synth_ct_chord(int N, int nang, int nbin, int r) {
    grid2d g; double px, py, dx, dy, t0, t1;
    ct_ray(N, nang, nbin, r, &g, &px, &py, &dx, &dy);
    if (!clip_line(&g, px, py, dx, dy, -1e30, 1e30, &t0, &t1)) return 0.0;
    return t1 - t0;
}

/* ------------------------------------------------------------ seismic ---- */
/* Straight rays between points (sx,sy) -> (rx,ry) through an nx x ny grid of
 * square cells of size h with origin (0,0); cell index iy*nx + ix. */
int64_t synth_segments_count(int nx, int ny, double h, int64_t nrays, const double* seg,
                             int32_t* row_len) {
    int64_t tot = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : tot)
    for (int64_t r = 0; r < nrays; ++r) {
        grid2d g = {nx, ny, 0.0, 0.0, h, h};
        double x0 = seg[4 * r], y0 = seg[4 * r + 1], x1 = seg[4 * r + 2], y1 = seg[4 * r + 3];
        double L = hypot(x1 - x0, y1 - y0);
        int c = 0;
        if (L > 0) c = trace(&g, x0, y0, (x1 - x0) / L, (y1 - y0) / L, 0.0, L, NULL, NULL, 0);
        row_len[r] = c;
        tot += c;
    }
    return tot;
}

void synth_segments_fill(int nx, int ny, double h, int64_t nrays, const double* seg,
                         const int64_t* row_ptr, int32_t* col, float* val) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nrays; ++r) {
        grid2d g = {nx, ny, 0.0, 0.0, h, h};
        double x0 = seg[4 * r], y0 = seg[4 * r + 1], x1 = seg[4 * r + 2], y1 = seg[4 * r + 3];
        double L = hypot(x1 - x0, y1 - y0);
        int cap = (int)(row_ptr[r + 1] - row_ptr[r]);
        if (L > 0)
            trace(&g, x0, y0, (x1 - x0) / L, (y1 - y0) / L, 0.0, L, col + row_ptr[r],
                  val + row_ptr[r], cap);
    }
}

/* ------------------------------------------------------- radiotherapy ---- */
/* Pencil-beam dose influence.  Voxel grid nx x ny x nz of cubic voxels of
 * size vs, centred on the isocentre; voxel index (iz*ny + iy)*nx + ix.
 * nbeam coplanar beams at angles beam_deg[b] in the x-y plane.  Beam b has an
 * ns x nzb beamlet grid in its beam's-eye view (lateral axis w = (-sin, cos, 0),
 * axial axis z) with pitches ds, dz, centred on the isocentre; beamlet
 * (q, p) has column b*ns*nzb + q*ns + p.  Dose of beamlet to voxel:
 *   exp(-mu * depth) * exp(-r^2 / (2 sigma^2))   if r < cutoff, else 0,
 * with depth the distance from the grid boundary along the beam direction and
 * r the distance of the voxel centre to the beamlet's central axis. */
typedef struct {
    int nx, ny, nz;
    double vs;
    int nbeam;
    const double* beam_deg;
    int ns, nzb;
    double ds, dz, mu, sigma, cutoff;
} rt_geom;

static int rt_voxel(const rt_geom* G, int32_t vox, int32_t* cols, float* vals, int cap) {
    int ix = vox % G->nx, iy = (vox / G->nx) % G->ny, iz = vox / (G->nx * G->ny);
    double px = (ix + 0.5 - 0.5 * G->nx) * G->vs;
    double py = (iy + 0.5 - 0.5 * G->ny) * G->vs;
    double pz = (iz + 0.5 - 0.5 * G->nz) * G->vs;
    double hx = 0.5 * G->nx * G->vs, hy = 0.5 * G->ny * G->vs;
    int cnt = 0;
    double inv2s2 = 1.0 / (2.0 * G->sigma * G->sigma);
    for (int b = 0; b < G->nbeam; ++b) {
        double th = G->beam_deg[b] * M_PI / 180.0;
        double ux = cos(th), uy = sin(th);
        /* depth: distance back along -u to the box boundary */
        double tb = INFINITY;
        if (ux > 0) tb = fmin(tb, (px + hx) / ux);
        if (ux < 0) tb = fmin(tb, (px - hx) / ux);
        if (uy > 0) tb = fmin(tb, (py + hy) / uy);
        if (uy < 0) tb = fmin(tb, (py - hy) / uy);
        double depth = tb;
        double att = exp(-G->mu * depth);
        double s = -px * uy + py * ux; /* lateral coordinate along w */
        double z = pz;
        double fp0 = 0.5 * (G->ns - 1), fq0 = 0.5 * (G->nzb - 1);
        int plo = (int)ceil((s - G->cutoff) / G->ds + fp0);
        int phi = (int)floor((s + G->cutoff) / G->ds + fp0);
        int qlo = (int)ceil((z - G->cutoff) / G->dz + fq0);
        int qhi = (int)floor((z + G->cutoff) / G->dz + fq0);
        if (plo < 0) plo = 0;
        if (phi > G->ns - 1) phi = G->ns - 1;
        if (qlo < 0) qlo = 0;
        if (qhi > G->nzb - 1) qhi = G->nzb - 1;
        for (int q = qlo; q <= qhi; ++q) {
            double dzq = z - (q - fq0) * G->dz;
            for (int p = plo; p <= phi; ++p) {
                double dsp = s - (p - fp0) * G->ds;
                double r2 = dsp * dsp + dzq * dzq;
                if (r2 >= G->cutoff * G->cutoff) continue;
                if (cols && cnt < cap) {
                    cols[cnt] = b * G->ns * G->nzb + q * G->ns + p;
                    vals[cnt] = (float)(att * exp(-r2 * inv2s2));
                }
                cnt++;
            }
        }
    }
    return cnt;
}

int64_t synth_rt_count(int nx, int ny, int nz, double vs, int nbeam, const double* beam_deg,
                       int ns, int nzb, double ds, double dz, double mu, double sigma,
                       double cutoff, int64_t nvox, const int32_t* voxels, int32_t* row_len) {
    rt_geom G = {nx, ny, nz, vs, nbeam, beam_deg, ns, nzb, ds, dz, mu, sigma, cutoff};
    int64_t tot = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : tot)
    for (int64_t r = 0; r < nvox; ++r) {
        int c = rt_voxel(&G, voxels[r], NULL, NULL, 0);
        row_len[r] = c;
        tot += c;
    }
    return tot;
}

void synth_rt_fill(int nx, int ny, int nz, double vs, int nbeam, const double* beam_deg, int ns,
                   int nzb, double ds, double dz, double mu, double sigma, double cutoff,
                   int64_t nvox, const int32_t* voxels, const int64_t* row_ptr, int32_t* col,
                   float* val) {
    rt_geom G = {nx, ny, nz, vs, nbeam, beam_deg, ns, nzb, ds, dz, mu, sigma, cutoff};
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < nvox; ++r) {
        int cap = (int)(row_ptr[r + 1] - row_ptr[r]);
        rt_voxel(&G, voxels[r], col + row_ptr[r], val + row_ptr[r], cap);
    }
}

/* Column indices from rt_voxel are increasing: beams in order, then q, then p. */

int synth_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
