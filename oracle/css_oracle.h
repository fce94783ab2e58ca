/*
 * css_oracle.h -- plain, slow, FP64 CPU oracle for the curved-surface MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only in the
 * seeded input generators.
 *
 * What it computes (paper sections in brackets):
 *   - intrinsic mesh preparation: per-face planar layouts, half-edge frames,
 *     vertex angle sums                                          [Sec. 2.2]
 *   - exact polyhedral geodesic distance and initial tangent from one source
 *     point to a list of target points, by continuous window propagation
 *     (the MMP family: unfold across each crossed edge, intersect windows,
 *     prune, stop at the cutoff) processed in a true priority order
 *                                                        [Sec. 2.2, Sec. 3.1]
 *   - neighbour lists with the Euclidean lower-bound prefilter   [Sec. 3.1]
 *   - forces  F_i = sum_j -U'(l_ij) * grad_i l_ij                [Sec. 3.1]
 *   - the straightest face-walk "shift" with parallel transport  [Sec. 3.2]
 *   - velocity Verlet NVE, Brownian and active Brownian updates  [Sec. 2.1]
 *   - Philox4x32-10 (Salmon et al., SC'11) + Box-Muller normals
 */
#ifndef CSS_ORACLE_H
#define CSS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct om_mesh om_mesh;

typedef struct {
    int64_t windows_created;      /* windows that survived insertion (incl. split pieces) */
    int64_t windows_propagated;   /* windows unfolded into their next face */
    int64_t windows_dropped;      /* candidate windows fully dominated on insertion */
    int64_t vertex_events;        /* pseudo-source vertex emissions */
    int64_t sources;              /* sources processed */
    int64_t queries;              /* target evaluations */
} om_stats;

typedef struct { int32_t kind; double eps, sigma, r_cut, A; } om_potential;      /* kind 0 harmonic, 1 WCA, 2 Gaussian */
typedef struct { int32_t kind; double dt, kT, lam, v0, Dr, mass, max_disp; } om_integrator; /* kind 0 NVE, 1 BD, 2 ABP, 3 GD, 4 FIRE */

/* FIRE constants (the published defaults) */
#define OM_FIRE_ALPHA0 0.1
#define OM_FIRE_FINC 1.1
#define OM_FIRE_FDEC 0.5
#define OM_FIRE_FALPHA 0.99
#define OM_FIRE_NMIN 5
#define OM_FIRE_DTMAX 10.0   /* times the initial dt */

/* mesh: X (nv x 3), F (nf x 3, CCW outward), period NULL or {Lx, Ly}.  Returns 0 or <0. */
int  om_mesh_create(const double* X, int64_t nv, const int32_t* F, int64_t nf,
                    const double* period, om_mesh** out);
void om_mesh_destroy(om_mesh* m);
int64_t om_mesh_num_edges(const om_mesh* m);
void om_mesh_vertex_info(const om_mesh* m, double* theta, uint8_t* pseudo, uint8_t* boundary);
void om_face_frame(const om_mesh* m, int32_t f, double* out9);          /* origin, e1, e2 */
void om_world_position(const om_mesh* m, int32_t f, const double* bary, double* out3);

/* Geodesic distance/tangent from source (f0, bary0) to nt targets.  Targets farther
 * than r_c (or unreachable) get dist = +INF and tangent 0.  r_c may be +INF. */
int om_geodesic_query(const om_mesh* m, int32_t f0, const double* bary0, double r_c,
                      int64_t nt, const int32_t* tf, const double* tb,
                      double* dist, double* tan3, om_stats* st);

/* Ordered pairs (i, j), i != j, with l_ij < r_c.  CSR rows in source order, columns in
 * increasing j.  If cap < needed, returns -5 and sets *n_pairs to the needed count. */
int om_neighbors(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
                 double r_c, int64_t cap, int64_t* n_pairs, int64_t* row_start,
                 int32_t* nbr_j, double* dist, double* tan3, int nthreads, om_stats* st);

/* Same pairs for a subset of sources only (rows for src[0..ns)). */
int om_neighbors_subset(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
                        double r_c, int64_t ns, const int64_t* src, int64_t cap,
                        int64_t* n_pairs, int64_t* row_start, int32_t* nbr_j, double* dist,
                        double* tan3, int nthreads, om_stats* st);

/* As om_neighbors_subset, plus gap[pair]: how much longer the shortest candidate path
 * with a different initial tangent is (+INF if none).  A small gap marks a point near
 * the cut locus, where the tangent is set-valued and any tiny error may switch it. */
int om_neighbors_gap(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
                     double r_c, int64_t ns, const int64_t* src, int64_t cap,
                     int64_t* n_pairs, int64_t* row_start, int32_t* nbr_j, double* dist,
                     double* tan3, double* gap, int nthreads, om_stats* st);

double om_pair_energy(const om_potential* p, double l);       /* U(l) */
double om_pair_dudl(const om_potential* p, double l);         /* dU/dl */

/* F (n x 3, world, in each particle's face plane) and E_pot = 1/2 sum_ij U(l_ij). */
int om_forces(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
              double r_c, const om_potential* pot, double* F, double* epot, int nthreads);
/* Forces on the listed particles src[0..ns) only (src NULL: particles 0..ns-1): F is ns x 3,
   e_src (ns, or NULL) receives each listed particle's half pair energies 1/2 sum_j U(l_ij). */
int om_forces_subset(const om_mesh* m, int64_t n, const int32_t* face, const double* bary, double r_c,
                     const om_potential* pot, int64_t ns, const int64_t* src, double* F, double* e_src,
                     int nthreads);

/* Shift one particle by the world tangent displacement disp3 along the surface,
 * carrying ncarry world tangent vectors (parallel transport).  Returns the number of
 * edge crossings (>= 0) or <0 on error. */
int om_shift(const om_mesh* m, int32_t* face, double* bary, const double* disp3,
             int ncarry, double* carry3);
/* The straightest walk of om_shift as a polyline (start, each crossing, end; world
 * positions, at most cap points, *npts = all of them); face/bary become the end point. */
int om_trace(const om_mesh* m, int32_t* face, double* bary, const double* disp3, int cap, double* pts,
             int* npts);

/* Shortest paths of np pairs (src[p] -> dst[p]) as polylines (Sec. 2.2: straight legs in
 * the unfolding that meet at pseudo-source vertices), rebuilt from the links the window
 * propagation records: the source point, every edge crossing and bend vertex, the target
 * (world positions, wrapped into the period on periodic meshes; at most cap points per
 * pair in pts[p*cap*3 ...], npts[p] = all of them, 0 when l >= r_c).  nlegs[p] = straight
 * legs, dist[p] = l, gap[p] = the largest distance between a leg walk's end and the node
 * it must reach.  Pairs sorted by src reuse one propagation. */
int om_geodesic_paths(const om_mesh* m, int64_t n, const int32_t* face, const double* bary, double r_c,
                      int64_t np, const int32_t* src, const int32_t* dst, int cap, double* pts, int32_t* npts,
                      int32_t* nlegs, double* dist, double* gap);

/* nsteps of the chosen dynamics.  vel used by NVE, orient by ABP, force in/out (the
 * force at the current positions must be valid on entry for NVE).  noise: NULL, or
 * nsteps*n*2 standard normals used instead of the Philox stream. */
int om_integrate(const om_mesh* m, int64_t n, int32_t* face, double* bary, double* vel,
                 double* orient, double* force, const om_potential* pot,
                 const om_integrator* it, double r_c, int64_t nsteps, uint64_t seed,
                 int64_t step0, const double* noise, double* epot, int nthreads);

void om_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* FIRE minimisation steps (see css_oracle.c); state[3] = {dt, alpha, steps with P > 0}. */
int om_fire(const om_mesh* m, int64_t n, int32_t* face, double* bary, double* vel, double* force,
            const om_potential* pot, const om_integrator* it, double r_c, int64_t nsteps, double* state,
            double* epot, int nthreads);
void om_normal_pair(uint64_t seed, uint64_t particle, uint64_t step, double* z0, double* z1);

#ifdef __cplusplus
}
#endif
#endif
