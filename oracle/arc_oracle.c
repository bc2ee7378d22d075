/*
 * arc_oracle.c -- FP64 CPU oracle for the ARC hot path (tracer + chemistry).
 *
 * TEST INFRASTRUCTURE ONLY (see arc_oracle.h).  Plain, single-threaded,
 * recursive, written to be checked by eye against the paper:
 *   Hartley & Ricotti, "ARC: Adaptive Ray-tracing with CUDA" (arXiv 1807.07094).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared arc_oracle.c -lm
 */
#include "arc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define KB 1.380649e-16          /* erg/K */
#define EVERG 1.602176634e-12    /* erg per eV */
#define ORC_MAXSUB 100000
#define TFLOOR 1.0

static const double E_S[3] = {13.6, 24.6, 54.4};   /* HI, HeI, HeII edges [eV] */

/* ------------------------------------------------------------------------- */
/* HEALPix, nested scheme (Sec. 2.1: ray directions; Gorski et al. 2005).     */
/* A level-l map has nside = 2^l and 12 nside^2 equal-area pixels; pixel p of */
/* level l has the children 4p..4p+3 at level l+1.                            */
/* ------------------------------------------------------------------------- */

/* face layout of the 12 base pixels: ring offset and longitude offset */
static const int FACE_RING[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int FACE_LON[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

static void split_bits(uint64_t ipf, int level, int64_t* ix, int64_t* iy) {
    int64_t x = 0, y = 0;
    for (int b = 0; b < level; b++) {
        x |= (int64_t)((ipf >> (2 * b)) & 1u) << b;
        y |= (int64_t)((ipf >> (2 * b + 1)) & 1u) << b;
    }
    *ix = x;
    *iy = y;
}

static uint64_t join_bits(int64_t ix, int64_t iy, int level) {
    uint64_t p = 0;
    for (int b = 0; b < level; b++) {
        p |= (uint64_t)((ix >> b) & 1) << (2 * b);
        p |= (uint64_t)((iy >> b) & 1) << (2 * b + 1);
    }
    return p;
}

void orc_pix2vec_nest(int level, uint64_t pix, double v[3]) {
    const int64_t ns = (int64_t)1 << level;
    const int64_t npface = ns * ns;
    const int face = (int)(pix / (uint64_t)npface);
    int64_t ix, iy;
    split_bits(pix % (uint64_t)npface, level, &ix, &iy);

    /* ring index counted from the north pole, 1 .. 4 ns - 1 */
    const int64_t jr = FACE_RING[face] * ns - ix - iy - 1;
    int64_t nr;          /* pixels in the ring / 4 */
    int kshift;          /* equatorial rings alternate a half-pixel shift */
    double z, one_minus_z_or_plus = 0.0;
    int cap = 0;
    if (jr < ns) {                    /* north polar cap */
        nr = jr;
        one_minus_z_or_plus = (double)(nr * nr) / (3.0 * (double)npface);  /* 1 - z */
        z = 1.0 - one_minus_z_or_plus;
        kshift = 0;
        cap = 1;
    } else if (jr > 3 * ns) {         /* south polar cap */
        nr = 4 * ns - jr;
        one_minus_z_or_plus = (double)(nr * nr) / (3.0 * (double)npface);  /* 1 + z */
        z = one_minus_z_or_plus - 1.0;
        kshift = 0;
        cap = 1;
    } else {                          /* equatorial belt */
        nr = ns;
        z = (double)(2 * ns - jr) * 2.0 / (3.0 * (double)ns);
        kshift = (int)((jr - ns) & 1);
    }
    int64_t jp = (FACE_LON[face] * nr + ix - iy + 1 + kshift) / 2;
    if (jp > 4 * ns) jp -= 4 * ns;
    if (jp < 1) jp += 4 * ns;
    const double phi = ((double)jp - 0.5 * (double)(kshift + 1)) * (0.5 * PI) / (double)nr;
    double st;
    if (cap) {
        const double a = one_minus_z_or_plus;   /* sin^2 = a (2 - a) */
        st = sqrt(a * (2.0 - a));
    } else {
        st = sqrt((1.0 - z) * (1.0 + z));
    }
    v[0] = st * cos(phi);
    v[1] = st * sin(phi);
    v[2] = z;
}

uint64_t orc_vec2pix_nest(int level, const double v[3]) {
    const int64_t ns = (int64_t)1 << level;
    const double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double z = v[2] / len, za = fabs(z);
    double phi = atan2(v[1], v[0]);
    if (phi < 0.0) phi += 2.0 * PI;
    double tt = phi / (0.5 * PI);
    if (tt >= 4.0) tt -= 4.0;
    int face;
    int64_t ix, iy;
    if (za <= 2.0 / 3.0) {
        /* equatorial: index along the two families of pixel edge lines */
        const double t1 = (double)ns * (0.5 + tt);
        const double t2 = (double)ns * z * 0.75;
        const int64_t jp = (int64_t)(t1 - t2);
        const int64_t jm = (int64_t)(t1 + t2);
        const int64_t ifp = jp / ns, ifm = jm / ns;
        if (ifp == ifm) face = (int)(ifp | 4);
        else if (ifp < ifm) face = (int)ifp;
        else face = (int)(ifm + 8);
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - 1;
    } else {
        int ntt = (int)tt;
        if (ntt > 3) ntt = 3;
        const double tp = tt - ntt;
        const double tmp = (double)ns * sqrt(3.0 * (1.0 - za));
        int64_t jp = (int64_t)(tp * tmp);
        int64_t jm = (int64_t)((1.0 - tp) * tmp);
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (z >= 0) {
            face = ntt;
            ix = ns - jm - 1;
            iy = ns - jp - 1;
        } else {
            face = ntt + 8;
            ix = jp;
            iy = jm;
        }
    }
    return (uint64_t)face * (uint64_t)(ns * ns) + join_bits(ix, iy, level);
}

/* ------------------------------------------------------------------------- */
/* Split distance (Sec. 2.4, Fig. 1): a level-l ray covers the solid angle    */
/* Omega_l = 4 pi / (12 4^l); at distance r it meets 1 / (Omega_l r^2) rays   */
/* per unit cell face.  The ray splits where that falls to phi:               */
/*   r_split(l) = 1 / sqrt(phi Omega_l)   [cells].                            */
/* ------------------------------------------------------------------------- */
double orc_r_split(const orc_params* p, int level) {
    const double omega = 4.0 * PI / (12.0 * pow(4.0, level));
    return 1.0 / sqrt(p->phi * omega);
}

/* ------------------------------------------------------------------------- */
/* Ray tracing (Sec. 2.1 step iii, Sec. 2.4).                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_params* p;
    const double *nH, *xHI, *xHeI, *xHeII;
    int n;
    double dx, V, y;
    double *gamma, *heat;
    double absorbed, escaped;
    orc_ray_rec* recs;
    int64_t rec_cap, nrec, nseg;
    int overflow;
    const double* o;      /* current source position */
    uint32_t isrc;
    double thr_base;      /* term_frac * photons of one ray at l_base */
    double* cmargin;      /* optional: per cell, smallest face-tie margin of the
                             geometric corrections that touched it [cells] */
    /* Sec. 2.6: a ray's length while its optical depth in the softest group
     * is below 0.1; the minimum over the current source's rays */
    int soft;             /* softest group (lowest photon energy) */
    double rthin;         /* running minimum for the current source [cells] */
} tctx;

#define THIN_TAU 0.1      /* Sec. 2.6 */

/* absorber densities n_HI, n_HeI, n_HeII of a cell [cm^-3] (Sec. 2.3) */
static void absorbers(const tctx* c, int64_t idx, double ns[3]) {
    const double nh = c->nH[idx];
    ns[0] = nh * c->xHI[idx];
    ns[1] = c->y * nh * c->xHeI[idx];
    ns[2] = c->y * nh * c->xHeII[idx];
}

/* Deposit a photon rate A (group b) absorbed in cell idx into the per-absorber
 * rates.  Eq. (ion): the species share of A is dtau_{s,b}/dtau_b and the rate
 * per absorber is A_{s,b} / (V n_s); with dtau_{s,b} = sigma_{s,b} n_s L this is
 * A sigma_{s,b} L / (dtau_b V), which stays defined as n_s -> 0 (L = ds dx).
 * With kappa_b = dtau_b / ds, the optical depth per cell length, this is
 * A sigma_{s,b} dx / (kappa_b V), independent of the segment length. */
static void deposit(tctx* c, int64_t idx, int b, double A, double kappa_b) {
    const orc_params* p = c->p;
    const int64_t n3 = (int64_t)c->n * c->n * c->n;
    for (int s = 0; s < 3; s++) {
        if (p->sigma[s][b] <= 0.0) continue;
        const double rate = A * p->sigma[s][b] * c->dx / (kappa_b * c->V);   /* 1/s per absorber */
        c->gamma[s * n3 + idx] += rate;
        c->heat[s * n3 + idx] += rate * (p->E_group_eV[b] - E_S[s]) * EVERG;   /* Sec. 2.8 */
    }
}

/* tau0: optical depth in the softest group accumulated from where the ray's
 * ancestors started (Sec. 2.6); only the thin radius uses it. */
static void trace_ray(tctx* c, int level, uint64_t pix, double r0, const double* Nin, double tau0) {
    const orc_params* p = c->p;
    const int G = p->ngroups, n = c->n;
    double N[ORC_MAXG];
    for (int b = 0; b < G; b++) N[b] = Nin[b];

    double u[3];
    orc_pix2vec_nest(level, pix, u);
    const double r_stop = (level < p->l_max) ? orc_r_split(p, level) : INFINITY;
    const double thr = c->thr_base / pow(4.0, level - p->l_base);
    const double* o = c->o;

    int cell[3];
    double geo = INFINITY, term = INFINITY, exitm = INFINITY;
    for (int a = 0; a < 3; a++) {
        const double x = o[a] + r0 * u[a];
        cell[a] = (int)floor(x);
        if (r0 > 0.0) geo = fmin(geo, fabs(x - nearbyint(x)));
    }
    int visits = 0, end;
    double r = r0;
    int64_t idx = 0;
    double kap[ORC_MAXG] = {0};

    if (cell[0] < 0 || cell[0] >= n || cell[1] < 0 || cell[1] >= n || cell[2] < 0 || cell[2] >= n) {
        for (int b = 0; b < G; b++) c->escaped += N[b];
        if (tau0 < THIN_TAU) c->rthin = fmin(c->rthin, r0);
        end = ORC_END_ESCAPE;
        goto record;
    }
    /* a ray that starts at or beyond its split distance (rays launched at the
     * optically thin radius, Sec. 2.6) splits at once without a segment */
    if (isfinite(r_stop)) exitm = fmin(exitm, fabs(r0 - r_stop));
    if (r0 >= r_stop) {
        end = ORC_END_SPLIT;
        goto record;
    }
    for (;;) {
        /* distance to the next X, Y and Z cell boundary */
        double tn[3];
        for (int a = 0; a < 3; a++) {
            if (u[a] > 0.0) tn[a] = ((double)cell[a] + 1.0 - o[a]) / u[a];
            else if (u[a] < 0.0) tn[a] = ((double)cell[a] - o[a]) / u[a];
            else tn[a] = INFINITY;
        }
        int ax = 0;
        if (tn[1] < tn[ax]) ax = 1;
        if (tn[2] < tn[ax]) ax = 2;
        const double t = tn[ax];
        const int split = (r_stop <= t);
        const double r1 = split ? r_stop : t;
        double ds = r1 - r;
        if (ds < 0.0) ds = 0.0;
        if (isfinite(r_stop)) {
            geo = fmin(geo, fabs(t - r_stop));
            const int nxt = cell[ax] + ((u[ax] > 0.0) ? 1 : -1);
            if (nxt < 0 || nxt >= n) exitm = fmin(exitm, fabs(t - r_stop));
        }
        /* a face crossed right after a child's start is an undecided tie */
        if (visits == 0 && r0 > 0.0) geo = fmin(geo, ds);

        /* Eq. (ion): absorb in every group */
        idx = ((int64_t)cell[0] * n + cell[1]) * n + cell[2];
        double ns[3];
        absorbers(c, idx, ns);
        const double L = ds * c->dx;

        /* Sec. 2.5, Eq. (correction): the ray stands for a cone of width
         * L_pix = r sqrt(Omega_l) at the segment's midpoint; when that point is
         * closer than L_pix / 2 to the nearest face of the cell, only the
         * fraction f_c = 1/2 + D_edge / L_pix of the absorption stays in the
         * cell and 1 - f_c goes to the neighbour across that face
         * (Eq. correction2, read as photons: the neighbour takes them with its
         * own absorber shares, so the photon count is unchanged). */
        double fc = 1.0;
        int64_t nidx = -1;
        double nkap[ORC_MAXG] = {0};
        if (p->geo_corr && ds > 0.0) {
            const double rm = 0.5 * (r + r1);
            double dmin = INFINITY, d2 = INFINITY;
            int nax = 0, nside = 0, aax = 0, aside = 0;
            for (int a = 0; a < 3; a++) {
                const double f = o[a] + rm * u[a] - (double)cell[a];   /* position inside the cell */
                const double dd[2] = {f, 1.0 - f};
                for (int k = 0; k < 2; k++) {
                    if (dd[k] < dmin) {
                        d2 = dmin; aax = nax; aside = nside;
                        dmin = dd[k]; nax = a; nside = k ? 1 : -1;
                    } else if (dd[k] < d2) {
                        d2 = dd[k]; aax = a; aside = k ? 1 : -1;
                    }
                }
            }
            if (dmin < 0.0) dmin = 0.0;
            const double lpix = rm * sqrt(4.0 * PI / (12.0 * pow(4.0, level)));   /* width: sqrt of Omega_l */
            if (c->cmargin && dmin < 0.5 * lpix) {
                /* which face is nearest is a discontinuous decision: note how
                 * close it was in the cells whose deposit depends on it */
                const double mg = d2 - dmin;
                int alt[3] = {cell[0], cell[1], cell[2]}, nn[3] = {cell[0], cell[1], cell[2]};
                alt[aax] += aside;
                nn[nax] += nside;
                c->cmargin[idx] = fmin(c->cmargin[idx], mg);
                if (nn[nax] >= 0 && nn[nax] < n)
                    c->cmargin[((int64_t)nn[0] * n + nn[1]) * n + nn[2]] =
                        fmin(c->cmargin[((int64_t)nn[0] * n + nn[1]) * n + nn[2]], mg);
                if (alt[aax] >= 0 && alt[aax] < n)
                    c->cmargin[((int64_t)alt[0] * n + alt[1]) * n + alt[2]] =
                        fmin(c->cmargin[((int64_t)alt[0] * n + alt[1]) * n + alt[2]], mg);
            }
            int nb[3] = {cell[0], cell[1], cell[2]};
            nb[nax] += nside;
            if (p->geo_corr >= 2 && dmin < 0.5 * lpix) {
                /* Sec. 3.6 variants: the primary factor alone (linear, or squared
                 * as in the method it modifies); the rest of the absorbed photons
                 * is credited to no cell */
                fc = 0.5 + dmin / lpix;
                if (p->geo_corr == 3) fc = fc * fc;
            } else if (dmin < 0.5 * lpix && nb[nax] >= 0 && nb[nax] < n) {
                fc = 0.5 + dmin / lpix;
                nidx = ((int64_t)nb[0] * n + nb[1]) * n + nb[2];
                double nns[3];
                absorbers(c, nidx, nns);
                for (int b = 0; b < G; b++) {
                    double kb = 0.0;
                    for (int s = 0; s < 3; s++) kb += p->sigma[s][b] * nns[s];
                    nkap[b] = kb * c->dx;
                }
            }
        }
        for (int b = 0; b < G; b++) {
            double kb = 0.0;
            for (int s = 0; s < 3; s++) kb += p->sigma[s][b] * ns[s];
            kap[b] = kb * c->dx;              /* optical depth per cell length */
            const double dtau = kb * L;
            if (dtau > 0.0) {
                const double A = N[b] * (-expm1(-dtau));
                N[b] -= A;
                c->absorbed += A;
                if (nidx >= 0 && nkap[b] > 0.0) {
                    /* a neighbour without absorbers of this group takes nothing */
                    deposit(c, idx, b, fc * A, kap[b]);
                    deposit(c, nidx, b, (1.0 - fc) * A, nkap[b]);
                } else if (p->geo_corr >= 2) {
                    deposit(c, idx, b, fc * A, kap[b]);
                } else {
                    deposit(c, idx, b, A, kap[b]);
                }
            }
        }
        /* Sec. 2.6: where the softest group's optical depth reaches 0.1 */
        {
            double ks = 0.0;
            for (int s = 0; s < 3; s++) ks += p->sigma[s][c->soft] * ns[s];
            const double dt0 = ks * L;
            if (tau0 < THIN_TAU && tau0 + dt0 >= THIN_TAU)
                c->rthin = fmin(c->rthin, r + (THIN_TAU - tau0) / (ks * c->dx));
            tau0 += dt0;
        }
        visits++;
        c->nseg++;
        r = r1;

        double sumN = 0.0;
        for (int b = 0; b < G; b++) sumN += N[b];
        term = fmin(term, fabs(sumN - thr) / thr);
        if (sumN < thr) {
            /* terminate: the remaining photons go into this cell with its
             * species shares, so that no photon is lost (Sec. 2.4). */
            for (int b = 0; b < G; b++) {
                if (N[b] > 0.0) {
                    c->absorbed += N[b];
                    if (kap[b] > 0.0) deposit(c, idx, b, N[b], kap[b]);
                    N[b] = 0.0;
                }
            }
            if (tau0 < THIN_TAU) c->rthin = fmin(c->rthin, r);
            end = ORC_END_TERM;
            break;
        }
        if (split) {
            /* a face crossed right before the split distance is a near tie */
            geo = fmin(geo, ds);
            end = ORC_END_SPLIT;
            break;
        }
        cell[ax] += (u[ax] > 0.0) ? 1 : -1;
        if (cell[ax] < 0 || cell[ax] >= n) {
            /* leaving the box: radiation is lost (Sec. 3.5) */
            /* the exit face against the other faces: the one crossed just
             * before (this segment's length) and the ones just after */
            geo = fmin(geo, ds);
            for (int a = 0; a < 3; a++)
                if (a != ax) geo = fmin(geo, fabs(tn[a] - t));
            for (int b = 0; b < G; b++) c->escaped += N[b];
            if (tau0 < THIN_TAU) c->rthin = fmin(c->rthin, r);
            end = ORC_END_ESCAPE;
            break;
        }
    }
record:
    if (c->recs) {
        if (c->nrec < c->rec_cap) {
            orc_ray_rec* q = &c->recs[c->nrec];
            q->src = c->isrc;
            q->level = level;
            q->pix = pix;
            q->visits = visits;
            q->end = end;
            q->r0 = r0;
            q->r1 = r;
            q->geo_margin = geo;
            q->term_margin = term;
            q->exit_margin = exitm;
        } else {
            c->overflow = 1;
        }
    }
    c->nrec++;
    if (end == ORC_END_SPLIT) {
        /* four children at the next level, same radius, a quarter of the
         * photons each (Sec. 2.1 step iii.c) */
        double Nc[ORC_MAXG];
        for (int b = 0; b < G; b++) Nc[b] = N[b] / 4.0;
        for (int k = 0; k < 4; k++) trace_ray(c, level + 1, 4 * pix + (uint64_t)k, r, Nc, tau0);
    }
}

int orc_trace(const orc_params* p, const double* nH, const double* xHI,
              const double* xHeI, const double* xHeII,
              int nsrc, const double* pos, const double* ndot,
              double* gamma, double* heat, double* budget,
              orc_ray_rec* recs, int64_t rec_cap, int64_t* nrec, int64_t* nseg) {
    return orc_trace_ex(p, nH, xHI, xHeI, xHeII, nsrc, pos, ndot, gamma, heat, budget, recs, rec_cap, nrec,
                        nseg, NULL);
}

int orc_trace_ex(const orc_params* p, const double* nH, const double* xHI,
                 const double* xHeI, const double* xHeII,
                 int nsrc, const double* pos, const double* ndot,
                 double* gamma, double* heat, double* budget,
                 orc_ray_rec* recs, int64_t rec_cap, int64_t* nrec, int64_t* nseg, double* corr_margin) {
    orc_trace_opts o;
    memset(&o, 0, sizeof o);
    o.corr_margin = corr_margin;
    return orc_trace_opt(p, nH, xHI, xHeI, xHeII, nsrc, pos, ndot, gamma, heat, budget, recs, rec_cap, nrec,
                         nseg, &o);
}

/* Sec. 2.6, step 3: every cell whose centre lies within R of the source is
 * taken as exposed without absorption; the thin limit of Eq. (ion) for the
 * rays crossing it is S_b sigma_{s,b} / (4 pi r^2) per absorber, i.e. the cell
 * absorbs S_b kappa_b V / (4 pi r^2) photons per group (kappa_b per length).
 * r is the centre's distance from the source, floored at half a cell (the
 * paper gives no value in the source's own cell, where 1/r^2 diverges).
 * Returns the photons deposited. */
static double thin_fill(tctx* c, const double* o, double R, const double* S) {
    const orc_params* p = c->p;
    const int n = c->n, G = p->ngroups;
    double tot = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                const double dx = i + 0.5 - o[0], dy = j + 0.5 - o[1], dz = k + 0.5 - o[2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < R * R)) continue;
                const double rr = r2 > 0.25 ? r2 : 0.25;
                const int64_t idx = ((int64_t)i * n + j) * n + k;
                double ns[3];
                absorbers(c, idx, ns);
                for (int b = 0; b < G; b++) {
                    double kb = 0.0;
                    for (int s = 0; s < 3; s++) kb += p->sigma[s][b] * ns[s];
                    const double kap = kb * c->dx;   /* per cell length */
                    const double A = S[b] * kap / (4.0 * PI * rr);
                    if (A > 0.0) {
                        deposit(c, idx, b, A, kap);
                        tot += A;
                    }
                }
            }
    return tot;
}

int orc_trace_opt(const orc_params* p, const double* nH, const double* xHI,
                  const double* xHeI, const double* xHeII,
                  int nsrc, const double* pos, const double* ndot,
                  double* gamma, double* heat, double* budget,
                  orc_ray_rec* recs, int64_t rec_cap, int64_t* nrec, int64_t* nseg,
                  const orc_trace_opts* opt) {
    if (!p || p->n <= 0 || p->ngroups < 1 || p->ngroups > ORC_MAXG || p->l_base < 1 ||
        p->l_max < p->l_base || p->phi <= 0.0 || nsrc < 0 || !opt)
        return -1;
    if (opt->open && opt->r_start) return -1;   /* masks and the thin region do not combine */
    tctx c;
    memset(&c, 0, sizeof c);
    c.p = p;
    c.cmargin = opt->corr_margin;
    if (c.cmargin)
        for (int64_t i = 0; i < (int64_t)p->n * p->n * p->n; i++) c.cmargin[i] = INFINITY;
    c.nH = nH;
    c.xHI = xHI;
    c.xHeI = xHeI;
    c.xHeII = xHeII;
    c.n = p->n;
    c.dx = p->box_cm / p->n;
    c.V = c.dx * c.dx * c.dx;
    c.y = p->Y / (4.0 * (1.0 - p->Y));
    c.gamma = gamma;
    c.heat = heat;
    c.recs = recs;
    c.rec_cap = recs ? rec_cap : 0;
    c.soft = 0;
    for (int b = 1; b < p->ngroups; b++)
        if (p->E_group_eV[b] < p->E_group_eV[c.soft]) c.soft = b;
    const int64_t n3 = (int64_t)p->n * p->n * p->n;
    memset(gamma, 0, sizeof(double) * 3 * n3);   /* Sec. 2.1 step i */
    memset(heat, 0, sizeof(double) * 3 * n3);
    const int G = p->ngroups;
    const double nrays = 12.0 * pow(4.0, p->l_base);
    double launched = 0.0, thin = 0.0;
    for (int s = 0; s < nsrc; s++) {
        double N0[ORC_MAXG], S[ORC_MAXG], tot = 0.0;
        for (int b = 0; b < G; b++) {
            S[b] = ndot[(int64_t)s * G + b];
            N0[b] = S[b] / nrays;   /* equal share per packet */
            tot += S[b];
        }
        if (opt->r_thin_out) opt->r_thin_out[s] = 0.0;
        if (!(tot > 0.0)) continue;
        c.o = &pos[3 * (int64_t)s];
        c.isrc = (uint32_t)s;
        c.thr_base = p->term_frac * tot / nrays;
        c.rthin = INFINITY;
        const double R = opt->r_start ? opt->r_start[s] : 0.0;
        if (R > 0.0) thin += thin_fill(&c, c.o, R, S);
        for (uint64_t q = 0; q < (uint64_t)nrays; q++) {
            if (opt->open && !opt->open[(int64_t)s * (int64_t)nrays + (int64_t)q]) {
                /* anisotropic escape (Sec. 2.2): this direction emits nothing */
                if (c.recs && c.nrec < c.rec_cap) {
                    orc_ray_rec* r = &c.recs[c.nrec];
                    memset(r, 0, sizeof *r);
                    r->src = c.isrc;
                    r->level = p->l_base;
                    r->pix = q;
                    r->end = ORC_END_BLOCKED;
                    r->r0 = r->r1 = R;
                    r->geo_margin = r->term_margin = r->exit_margin = INFINITY;
                } else if (c.recs) {
                    c.overflow = 1;
                }
                c.nrec++;
                continue;
            }
            launched += tot / nrays;
            trace_ray(&c, p->l_base, q, R, N0, 0.0);
        }
        if (opt->r_thin_out) opt->r_thin_out[s] = isfinite(c.rthin) ? c.rthin : 0.0;
    }
    if (budget) {
        budget[0] = launched;
        budget[1] = c.absorbed;
        budget[2] = c.escaped;
    }
    if (opt->thin_photons) *opt->thin_photons = thin;
    if (nrec) *nrec = c.nrec;
    if (nseg) *nseg = c.nseg;
    return c.overflow ? -2 : 0;
}

/* ------------------------------------------------------------------------- */
/* Chemistry and energy (Sec. 2.7, 2.8).                                     */
/* Rate fits: Hui & Gnedin (1997) case-B recombination, collisional          */
/* ionisation and recombination cooling; Cen (1992) collisional excitation,  */
/* dielectronic recombination and free-free Gaunt factor; Compton cooling    */
/* off the CMB from Thomson scattering.  Pinned against published atomic     */
/* physics, not against these fits (tests/test_oracle_rates.py): tabulated   */
/* case-B coefficients, an independent collisional-ionisation fit, the mean  */
/* energy per recombination, hydrogenic scaling, line and ionisation         */
/* energies, collision strengths and the free-free coefficient.              */
/* ------------------------------------------------------------------------- */
#define T_HI 157807.0
#define T_HEI 285335.0
#define T_HEII 631515.0

static double hg_alpha_b(double lam) {       /* HII, HeIII (x2): case B */
    return 2.753e-14 * pow(lam, 1.5) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
}
static double hg_recool_b(double T, double lam) {   /* erg cm^3/s */
    return 3.435e-30 * T * pow(lam, 1.970) / pow(1.0 + pow(lam / 2.250, 0.376), 3.720);
}

void orc_rates(const orc_params* p, double T, double out[6]) {
    const double lHI = 2.0 * T_HI / T, lHeI = 2.0 * T_HEI / T, lHeII = 2.0 * T_HEII / T;
    out[0] = (p->alpha_B_fixed > 0.0) ? p->alpha_B_fixed : hg_alpha_b(lHI);
    out[1] = 1.26e-14 * pow(lHeI, 0.750) +
             1.90e-3 * pow(T, -1.5) * exp(-4.7e5 / T) * (1.0 + 0.3 * exp(-9.4e4 / T));
    out[2] = 2.0 * hg_alpha_b(lHeII);
    if (p->coll_ion) {
        const double t32 = pow(T, -1.5);
        out[3] = 21.11 * t32 * exp(-0.5 * lHI) * pow(lHI, -1.089) /
                 pow(1.0 + pow(lHI / 0.354, 0.874), 1.101);
        out[4] = 32.38 * t32 * exp(-0.5 * lHeI) * pow(lHeI, -1.146) /
                 pow(1.0 + pow(lHeI / 0.416, 0.987), 1.056);
        out[5] = 19.95 * t32 * exp(-0.5 * lHeII) * pow(lHeII, -1.089) /
                 pow(1.0 + pow(lHeII / 0.553, 0.735), 1.275);
    } else {
        out[3] = out[4] = out[5] = 0.0;
    }
}

/* Cooling terms [erg cm^-3 s^-1], one per process (ORC_NCOOL entries, order of
 * orc_cooling_terms in arc_oracle.h): collisional ionisation of HI, HeI, HeII;
 * recombination of HII (case B), HeII (radiative), HeIII (case B); dielectronic
 * recombination of HeII; collisional excitation of HI and HeII; free-free;
 * Compton scattering off the CMB. */
void orc_cooling_terms(const orc_params* p, double T, double nH, double nHI, double nHeI,
                       double nHeII, double ne, double L[ORC_NCOOL]) {
    const double y = p->Y / (4.0 * (1.0 - p->Y));
    const double nHe = y * nH;
    const double nHII = nH - nHI;
    double nHeIII = nHe - nHeI - nHeII;
    if (nHeIII < 0.0) nHeIII = 0.0;
    const double lHI = 2.0 * T_HI / T, lHeI = 2.0 * T_HEI / T, lHeII = 2.0 * T_HEII / T;
    double r[6];
    orc_rates(p, T, r);
    /* collisional ionisation: threshold energy per ionisation */
    L[0] = ne * r[3] * nHI * KB * T_HI;
    L[1] = ne * r[4] * nHeI * KB * T_HEI;
    L[2] = ne * r[5] * nHeII * KB * T_HEII;
    /* recombination (case B) and dielectronic recombination */
    L[3] = ne * hg_recool_b(T, lHI) * nHII;
    L[4] = ne * 1.26e-14 * pow(lHeI, 0.750) * KB * T * nHeII;
    /* HeIII is hydrogenic (Z = 2): Lambda(Z, T) = Z^3 Lambda_HII(T / Z^2), the
     * fit's temperature prefactor taken at the scaled temperature whose lambda
     * is lHeII */
    L[5] = ne * 8.0 * hg_recool_b(T * (T_HI / T_HEII), lHeII) * nHeIII;
    L[6] = ne * 1.24e-13 * pow(T, -1.5) * exp(-4.7e5 / T) * (1.0 + 0.3 * exp(-9.4e4 / T)) * nHeII;
    /* collisional excitation */
    const double sq = 1.0 + sqrt(T / 1e5);
    L[7] = ne * 7.5e-19 * exp(-118348.0 / T) / sq * nHI;
    L[8] = ne * 5.54e-17 * pow(T, -0.397) * exp(-473638.0 / T) / sq * nHeII;
    /* bremsstrahlung */
    const double lg = log10(T) - 5.5;
    const double gff = 1.1 + 0.34 * exp(-lg * lg / 3.0);
    L[9] = 1.42e-27 * gff * sqrt(T) * (nHII + nHeII + 4.0 * nHeIII) * ne;
    /* Compton scattering off the CMB: 4 sigma_T a k / (m_e c) T_g^4 (T - T_g) n_e */
    L[10] = 0.0;
    if (p->z_compton >= 0.0) {
        const double sigT = 6.6524587e-25, arad = 7.5657e-15, me = 9.1093837e-28, cl = 2.99792458e10;
        const double Tg = 2.725 * (1.0 + p->z_compton);
        L[10] = 4.0 * sigT * arad * KB / (me * cl) * Tg * Tg * Tg * Tg * (T - Tg) * ne;
    }
}

double orc_cooling(const orc_params* p, double T, double nH, double nHI, double nHeI,
                   double nHeII, double ne) {
    double L[ORC_NCOOL];
    orc_cooling_terms(p, T, nH, nHI, nHeI, nHeII, ne, L);
    double s = 0.0;
    for (int k = 0; k < ORC_NCOOL; k++) s += L[k];
    return s;
}

/* The sub-cycled update; min_sub > 0 also caps every sub-step at dt / min_sub
 * (a uniform refinement under which all species converge as min_sub grows;
 * the paper's limiter, min_sub = 0, controls only n_HI, n_HII and E). */
static int chem_subcycled(const orc_params* p, int64_t ncell, const double* nHa,
                          double* xHI, double* xHeI, double* xHeII, double* Ta,
                          const double* gamma, const double* heat, double dt, int min_sub,
                          int64_t* nsub_out) {
    const double y = p->Y / (4.0 * (1.0 - p->Y));
    const double eps = p->eps_sub;
    int capped = 0;
    int64_t nsub_total = 0;
    for (int64_t i = 0; i < ncell; i++) {
        const double nH = nHa[i];
        if (!(nH > 0.0)) continue;
        const double nHe = y * nH;
        double nHI = xHI[i] * nH, nHeI = xHeI[i] * nHe, nHeII = xHeII[i] * nHe, T = Ta[i];
        const double G0 = gamma[i], G1 = gamma[ncell + i], G2 = gamma[2 * ncell + i];
        const double H0 = heat[i], H1 = heat[ncell + i], H2 = heat[2 * ncell + i];
        double t = 0.0;
        int nsub = 0;
        for (;;) {
            if (nsub >= ORC_MAXSUB) {
                capped++;
                break;
            }
            /* electron density, Sec. 2.3 (He in HeII and HeIII) */
            const double ne = (nH - nHI) + nHeII + 2.0 * (nHe - nHeI - nHeII);
            double r[6];
            orc_rates(p, T, r);
            /* Eq. (anninos) for HI: dn/dt = D - C n with n_HII = nH - n_HI */
            const double DH = r[0] * ne * nH;
            const double CH = G0 + (r[3] + r[0]) * ne;
            const double dnHI = DH - CH * nHI;
            /* sub-cycle step: at most a fraction eps change of E, n_HI and
             * n_HII (the hydrogen densities floored at x_fp64 n_H) */
            double h = dt - t;
            int last = 1;
            if (min_sub > 0 && h > dt / min_sub) {
                h = dt / min_sub;
                last = 0;
            }
            const double lim = eps * fmax(fmin(nHI, nH - nHI), p->x_fp64 * nH);
            if (fabs(dnHI) * h > lim) {
                h = lim / fabs(dnHI);
                last = 0;
            }
            /* ... and of the helium densities n_HeI, n_HeII, n_HeIII (each
             * floored at x_fp64 n_He): Sec. 2.7 limits the change of every
             * quantity the equations track; the printed formula shows only the
             * pure-hydrogen pair */
            if (nHe > 0.0) {
                const double nHeIII = nHe - nHeI - nHeII;
                const double dHeI = r[1] * ne * nHeII - (G1 + r[4] * ne) * nHeI;
                const double dHeIII = (G2 + r[5] * ne) * nHeII - r[2] * ne * nHeIII;
                const double dHe[3] = {dHeI, -dHeI - dHeIII, dHeIII};
                const double nHeS[3] = {nHeI, nHeII, nHeIII};
                for (int k = 0; k < 3; k++) {
                    const double limk = eps * fmax(nHeS[k], p->x_fp64 * nHe);
                    if (fabs(dHe[k]) * h > limk) {
                        h = limk / fabs(dHe[k]);
                        last = 0;
                    }
                }
            }
            double E = 0.0, Edot = 0.0;
            if (!p->isothermal) {
                E = 1.5 * KB * T * (nH + nHe + ne);
                Edot = (nHI * H0 + nHeI * H1 + nHeII * H2) -
                       orc_cooling(p, T, nH, nHI, nHeI, nHeII, ne);
                if (fabs(Edot) * h > eps * E) {
                    h = eps * E / fabs(Edot);
                    last = 0;
                }
            }
            /* backward-difference update per species, ne frozen in the step */
            nHI = (nHI + h * DH) / (1.0 + h * CH);
            const double C1 = G1 + r[4] * ne, D1 = r[1] * ne * nHeII;
            nHeI = (nHeI + h * D1) / (1.0 + h * C1);
            if (nHeI > nHe) nHeI = nHe;
            const double C2 = G2 + (r[5] + r[1] + r[2]) * ne;
            const double D2 = (G1 + r[4] * ne) * nHeI + r[2] * ne * (nHe - nHeI);
            nHeII = (nHeII + h * D2) / (1.0 + h * C2);
            if (nHeII > nHe - nHeI) nHeII = nHe - nHeI;
            if (nHeII < 0.0) nHeII = 0.0;
            if (!p->isothermal) {
                const double ne1 = (nH - nHI) + nHeII + 2.0 * (nHe - nHeI - nHeII);
                T = (E + h * Edot) / (1.5 * KB * (nH + nHe + ne1));
                if (T < TFLOOR) T = TFLOOR;
            }
            nsub++;
            if (last) break;
            t += h;
        }
        nsub_total += nsub;
        xHI[i] = nHI / nH;
        if (nHe > 0.0) {
            xHeI[i] = nHeI / nHe;
            xHeII[i] = nHeII / nHe;
        }
        Ta[i] = T;
    }
    if (nsub_out) *nsub_out = nsub_total;
    return capped;
}

int orc_chem(const orc_params* p, int64_t ncell, const double* nHa,
             double* xHI, double* xHeI, double* xHeII, double* Ta,
             const double* gamma, const double* heat, double dt, int64_t* nsub_out) {
    return chem_subcycled(p, ncell, nHa, xHI, xHeI, xHeII, Ta, gamma, heat, dt, 0, nsub_out);
}

int orc_chem_refined(const orc_params* p, int64_t ncell, const double* nHa,
                     double* xHI, double* xHeI, double* xHeII, double* Ta,
                     const double* gamma, const double* heat, double dt, int min_sub,
                     int64_t* nsub_out) {
    if (min_sub < 1) return -1;
    return chem_subcycled(p, ncell, nHa, xHI, xHeI, xHeII, Ta, gamma, heat, dt, min_sub, nsub_out);
}

/* ------------------------------------------------------------------------- */
/* Radiative-transfer time step (Sec. 2.9), from the current state and the   */
/* rates of the last trace.  Per cell, with dn_HI/dt = alpha n_e n_HII -      */
/* (Gamma_HI + beta n_e) n_HI (Eq. anninos):                                  */
/*   dt_n = eps n_HI / |dn_HI/dt| over the cells with tau = n_HI sigma d > 0.5  */
/*   dt_I = eps / (sigma d |dn_HI/dt|)  over all cells                          */
/* with sigma the HI cross section of the lowest group and d the cell width;  */
/* out[0] = min dt_n, out[1] = min dt_I (+inf when no cell qualifies).        */
/* ------------------------------------------------------------------------- */
void orc_rt_timestep(const orc_params* p, int64_t ncell, const double* nHa, const double* xHI,
                     const double* xHeI, const double* xHeII, const double* Ta, const double* gamma,
                     double eps, double out[2]) {
    const double y = p->Y / (4.0 * (1.0 - p->Y));
    const double d = p->box_cm / p->n;
    const double sig = p->sigma[0][0];
    double dtn = INFINITY, dti = INFINITY;
    for (int64_t i = 0; i < ncell; i++) {
        const double nH = nHa[i];
        if (!(nH > 0.0)) continue;
        const double nHe = y * nH;
        const double nHI = xHI[i] * nH, nHeII = xHeII[i] * nHe;
        const double nHeIII = nHe - xHeI[i] * nHe - nHeII;
        const double n_e = (nH - nHI) + nHeII + 2.0 * nHeIII;   /* Sec. 2.3 */
        double r[6];
        orc_rates(p, Ta[i], r);
        const double rate = fabs(r[0] * n_e * (nH - nHI) - (gamma[i] + r[3] * n_e) * nHI);
        if (!(rate > 0.0)) continue;
        if (nHI * sig * d > 0.5) dtn = fmin(dtn, eps * nHI / rate);
        dti = fmin(dti, eps / (sig * d * rate));
    }
    out[0] = dtn;
    out[1] = dti;
}

