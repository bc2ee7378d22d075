/*
 * arc_oracle.h -- FP64 CPU oracle for the ARC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke entry and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path; it is the plain, slow,
 * single-threaded statement of what the path computes, used to check it.
 *
 * Sections of the paper it follows (Hartley & Ricotti, "ARC"):
 *   Sec. 2.1  program design: 48 HEALPix level-1 packets per source, split
 *             into 4 children at the next level, termination.
 *   Sec. 2.2  anisotropic escape: emitted rays of a source may be blocked.
 *   Sec. 2.4  photon transmission: cell-by-cell stepping to the next X/Y/Z
 *             boundary, Eq. (ion) photon-conserving absorption.
 *   Sec. 2.5  geometric correction f_c and its secondary f'_c.
 *   Sec. 2.6  optically thin approximation: radius R_{tau<0.1}, the thin
 *             fill inside it, rays launched at R.
 *   Sec. 2.3  grid data: electron density.
 *   Sec. 2.7  ionisation calculation: Eq. (diffeq), Eq. (anninos), the
 *             sub-cycle step limiter with epsilon = 0.1.
 *   Sec. 2.8  heating and cooling: photoheating h(nu - nu_S) s_nu n_SI.
 */
#ifndef ARC_ORACLE_H
#define ARC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXG 4

typedef struct {
    int    n;                      /* cells per side                                */
    double box_cm;                 /* side length [cm]                              */
    int    ngroups;                /* frequency groups, 1..ORC_MAXG                 */
    double E_group_eV[ORC_MAXG];   /* energy per photon of each group [eV]          */
    double sigma[3][ORC_MAXG];     /* sigma_{s,b} [cm^2], s = HI, HeI, HeII         */
    double Y;                      /* helium mass fraction                          */
    double phi;                    /* split when fewer than phi rays cross a face   */
    int    l_base;                 /* HEALPix level of the emitted packets (>= 1)   */
    int    l_max;                  /* deepest level; rays at l_max never split      */
    double term_frac;              /* terminate below this fraction of emission     */
    double eps_sub;                /* sub-cycle fractional-change limit (0.1)       */
    double x_fp64;                 /* neutral-fraction floor used by the limiter    */
    int    isothermal;             /* 1: T fixed, no energy equation                */
    double alpha_B_fixed;          /* > 0: constant HII case-B coefficient          */
    int    coll_ion;               /* 1: collisional ionisation on                  */
    double z_compton;              /* >= 0: Compton cooling off the CMB at this z   */
    int    geo_corr;               /* geometric correction (Sec. 2.5): 0 none; 1 f_c
                                      with the secondary f'_c to the nearest
                                      neighbour; 2 f_c alone; 3 f_c squared alone
                                      (the last two are the Sec. 3.6 comparison
                                      variants and do not conserve photons)       */
} orc_params;

/* end reasons of a ray */
#define ORC_END_SPLIT 1
#define ORC_END_ESCAPE 2
#define ORC_END_TERM 3
#define ORC_END_BLOCKED 4   /* a masked emission direction: no photons, no cells */

typedef struct {
    uint32_t src;        /* source index                                         */
    int32_t  level;      /* HEALPix level                                        */
    uint64_t pix;        /* nested pixel index at that level                     */
    int32_t  visits;     /* cell segments traced (zero-length ones included)     */
    int32_t  end;        /* ORC_END_*                                            */
    double   r0, r1;     /* start / end distance from the source [cells]         */
    double   geo_margin; /* smallest distance of a geometric decision that sets
                            this ray's own visit count to a tie [cells]         */
    double   term_margin;/* smallest |sum N - threshold| / threshold             */
    double   exit_margin;/* |t - r_split| for a box-exit face near the split
                            distance: decides whether children exist [cells]    */
} orc_ray_rec;

/* HEALPix nested scheme (Gorski et al. 2005): pixel centre -> unit vector. */
void orc_pix2vec_nest(int level, uint64_t pix, double v[3]);
/* unit vector (any length) -> nested pixel index. */
uint64_t orc_vec2pix_nest(int level, const double v[3]);

/* Split distance of a level-l ray [cells]. */
double orc_r_split(const orc_params* p, int level);

/*
 * One radiative-transfer pass over all sources (Sec. 2.1 steps i and iii).
 * Fields: n^3 doubles in C order [i][j][k], k fastest; position (x,y,z) maps
 * to (i,j,k) and cell (i,j,k) spans [i,i+1) x [j,j+1) x [k,k+1).
 * pos: nsrc*3 grid units.  ndot: nsrc*ngroups photons/s.
 * Outputs: gamma, heat: 3*n^3 (species-major), per absorber [1/s], [erg/s];
 * budget[0..2] = emitted, absorbed, escaped photons/s.
 * recs (may be NULL) receives one record per ray, up to rec_cap.
 * Returns 0 on success, -1 on bad arguments, -2 if recs overflowed.
 */
int orc_trace(const orc_params* p, const double* nH, const double* xHI,
              const double* xHeI, const double* xHeII,
              int nsrc, const double* pos, const double* ndot,
              double* gamma, double* heat, double* budget,
              orc_ray_rec* recs, int64_t rec_cap, int64_t* nrec, int64_t* nseg);
/* The same, and with corr_margin (n^3, may be NULL) also, per cell, the
 * smallest margin (second-nearest minus nearest face distance [cells]) of
 * the geometric-correction face choices whose deposits touched the cell. */
int orc_trace_ex(const orc_params* p, const double* nH, const double* xHI,
                 const double* xHeI, const double* xHeII,
                 int nsrc, const double* pos, const double* ndot,
                 double* gamma, double* heat, double* budget,
                 orc_ray_rec* recs, int64_t rec_cap, int64_t* nrec, int64_t* nseg, double* corr_margin);

/* Options of orc_trace_opt (each may be NULL / 0). */
typedef struct {
    double* corr_margin;        /* as for orc_trace_ex                                 */
    const double* r_start;      /* nsrc: optically thin radius R per source [cells]
                                   (Sec. 2.6): cells with centres within R get the
                                   thin-limit rate, rays start at distance R       */
    double* r_thin_out;         /* nsrc: min over the source's rays of the length
                                   while the softest group's optical depth, counted
                                   from the ray's start, is below 0.1 (0 if none)  */
    double* thin_photons;       /* photons/s deposited by the thin fill               */
    const unsigned char* open;  /* nsrc x 12*4^l_base: 0 blocks that emitted ray
                                   (anisotropic escape, Sec. 2.2); not with r_start */
} orc_trace_opts;

/* orc_trace with options.  budget[0] counts the photons of emitted (open)
 * rays only; the thin fill's photons are not part of budget[1]. */
int orc_trace_opt(const orc_params* p, const double* nH, const double* xHI,
                  const double* xHeI, const double* xHeII,
                  int nsrc, const double* pos, const double* ndot,
                  double* gamma, double* heat, double* budget,
                  orc_ray_rec* recs, int64_t rec_cap, int64_t* nrec, int64_t* nseg,
                  const orc_trace_opts* opt);

/*
 * Sub-cycled chemistry / energy update of ncell cells over dt seconds
 * (Sec. 2.7, 2.8).  xHI, xHeI, xHeII, T are updated in place.
 * gamma, heat: 3*ncell species-major (the layout orc_trace writes).
 * nsub (may be NULL) receives the total number of sub-steps.
 * Returns 0, or the number of cells that hit the sub-step cap.
 */
int orc_chem(const orc_params* p, int64_t ncell, const double* nH,
             double* xHI, double* xHeI, double* xHeII, double* T,
             const double* gamma, const double* heat, double dt, int64_t* nsub);

/* The same update with every sub-step also capped at dt / min_sub (min_sub
 * >= 1, else -1): a uniform refinement under which all species converge to
 * the solution of the rate equations as min_sub grows.  The paper's limiter
 * bounds only the changes of n_HI, n_HII and E per sub-step, so the helium
 * fractions of orc_chem carry the first-order error of the step it takes. */
int orc_chem_refined(const orc_params* p, int64_t ncell, const double* nH,
                     double* xHI, double* xHeI, double* xHeII, double* T,
                     const double* gamma, const double* heat, double dt, int min_sub,
                     int64_t* nsub);

/* Radiative-transfer time step (Sec. 2.9) from the current state and the HI
 * photoionisation rate of the last trace (gamma: ncell values):
 * out[0] = min over cells with n_HI sigma d > 0.5 of eps n_HI / |dn_HI/dt|,
 * out[1] = min over cells of eps / (sigma d |dn_HI/dt|); +inf if none. */
void orc_rt_timestep(const orc_params* p, int64_t ncell, const double* nH, const double* xHI,
                     const double* xHeI, const double* xHeII, const double* T, const double* gamma,
                     double eps, double out[2]);

/* Rate coefficients at temperature T (for tests):
 * out[0..5] = alpha_HII, alpha_HeII(+dielectronic), alpha_HeIII,
 *             beta_HI, beta_HeI, beta_HeII  [cm^3/s]. */
void orc_rates(const orc_params* p, double T, double out[6]);
/* Cooling rate Lambda [erg/s/cm^3] of a state: the sum of the terms below. */
double orc_cooling(const orc_params* p, double T, double nH, double nHI, double nHeI,
                   double nHeII, double ne);
/* The cooling terms one by one [erg/s/cm^3] (for tests): collisional ionisation
 * of HI, HeI, HeII; recombination of HII (case B), HeII (radiative), HeIII (case
 * B); dielectronic recombination of HeII; collisional excitation of HI, HeII;
 * free-free; Compton. */
#define ORC_NCOOL 11
void orc_cooling_terms(const orc_params* p, double T, double nH, double nHI, double nHeI,
                       double nHeII, double ne, double L[ORC_NCOOL]);

#ifdef __cplusplus
}
#endif
#endif
