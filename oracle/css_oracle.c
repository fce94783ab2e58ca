/*
 * css_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see css_oracle.h).
 *
 * Written for readability, not speed: a binary heap gives the exact priority
 * order, windows live in per-edge arrays, every window insertion is compared
 * against every window already on that edge.
 *
 * Conventions
 *   face f, corner k in {0,1,2}, half-edge h = 3f+k runs F[f][k] -> F[f][k+1];
 *   the face layout puts P0 = (0,0), P1 = (L01, 0), P2 = (x2, y2 > 0);
 *   the frame of half-edge h has its origin at P_k, x along the edge and +y
 *   pointing into face f.  A window stored on h "propagates into" face f: its
 *   pseudo-source s lies on the other side (s.y <= 0) and the distance it
 *   carries to a point X is sigma + |X - s| (Sec. 2.2: shortest paths are
 *   straight lines in planar unfoldings of face strips).
 */
#include "css_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OM_INF (1.0 / 0.0)
#define OM_PI 3.14159265358979323846

struct om_mesh {
    int64_t nv, nf, ne;
    double* X;
    int32_t* F;
    int periodic;
    double per[2];
    int32_t* twin;      /* per half-edge: opposite half-edge or -1 on the boundary */
    int32_t* edge;      /* per half-edge: undirected edge id */
    double* hl;         /* per half-edge: length */
    double* hcx;        /* per half-edge: opposite vertex in the half-edge frame */
    double* hcy;
    double* lay;        /* per face: L01, x2, y2 */
    double* frame;      /* per face: origin(3), e1(3), e2(3) */
    double* theta;      /* per vertex: sum of incident corner angles */
    uint8_t* bnd;
    uint8_t* pseudo;
    int32_t* ring_start;/* per vertex: corners h = 3f+k with F[h] == v */
    int32_t* ring;
};

/* ------------------------------------------------------------------ small 2D helpers */
static double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }
static double dot2(double ax, double ay, double bx, double by) { return ax * bx + ay * by; }

static void face_pt(const om_mesh* m, int64_t f, int k, double* x, double* y) {
    k %= 3;
    if (k == 0) { *x = 0.0; *y = 0.0; }
    else if (k == 1) { *x = m->lay[3 * f]; *y = 0.0; }
    else { *x = m->lay[3 * f + 1]; *y = m->lay[3 * f + 2]; }
}

/* point of face f given in the face layout -> coordinates in the frame of half-edge 3f+k */
static void to_he_frame(const om_mesh* m, int64_t f, int k, double px, double py, double* hx, double* hy) {
    double ax, ay, bx, by;
    face_pt(m, f, k, &ax, &ay);
    face_pt(m, f, k + 1, &bx, &by);
    double L = hypot(bx - ax, by - ay);
    double dx = (bx - ax) / L, dy = (by - ay) / L;
    *hx = dot2(px - ax, py - ay, dx, dy);
    *hy = cross2(dx, dy, px - ax, py - ay);
}

static void min_image(const om_mesh* m, double* d) {
    if (!m->periodic) return;
    for (int a = 0; a < 2; ++a) d[a] -= m->per[a] * floor(d[a] / m->per[a] + 0.5);
}

/* ------------------------------------------------------------------ mesh preparation (Sec. 2.2) */
typedef struct { int32_t a, b, h; } ekey;
static int ekey_cmp(const void* p, const void* q) {
    const ekey* x = (const ekey*)p; const ekey* y = (const ekey*)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return x->h < y->h ? -1 : (x->h > y->h);
}

int om_mesh_create(const double* X, int64_t nv, const int32_t* F, int64_t nf,
                   const double* period, om_mesh** out) {
    *out = NULL;
    if (nv <= 0 || nf <= 0) return -1;
    for (int64_t i = 0; i < 3 * nf; ++i) if (F[i] < 0 || F[i] >= nv) return -1;
    om_mesh* m = (om_mesh*)calloc(1, sizeof(om_mesh));
    m->nv = nv; m->nf = nf;
    m->X = (double*)malloc(sizeof(double) * 3 * nv); memcpy(m->X, X, sizeof(double) * 3 * nv);
    m->F = (int32_t*)malloc(sizeof(int32_t) * 3 * nf); memcpy(m->F, F, sizeof(int32_t) * 3 * nf);
    if (period) { m->periodic = 1; m->per[0] = period[0]; m->per[1] = period[1]; }
    int64_t nh = 3 * nf;
    m->twin = (int32_t*)malloc(sizeof(int32_t) * nh);
    m->edge = (int32_t*)malloc(sizeof(int32_t) * nh);
    m->hl = (double*)malloc(sizeof(double) * nh);
    m->hcx = (double*)malloc(sizeof(double) * nh);
    m->hcy = (double*)malloc(sizeof(double) * nh);
    m->lay = (double*)malloc(sizeof(double) * 3 * nf);
    m->frame = (double*)malloc(sizeof(double) * 9 * nf);
    m->theta = (double*)calloc(nv, sizeof(double));
    m->bnd = (uint8_t*)calloc(nv, 1);
    m->pseudo = (uint8_t*)calloc(nv, 1);

    /* undirected edges by sorting (min, max) vertex keys; manifold + orientation checks */
    ekey* K = (ekey*)malloc(sizeof(ekey) * nh);
    for (int64_t h = 0; h < nh; ++h) {
        int32_t a = F[h], b = F[3 * (h / 3) + (h % 3 + 1) % 3];
        if (a == b) { free(K); om_mesh_destroy(m); return -2; }
        K[h].a = a < b ? a : b; K[h].b = a < b ? b : a; K[h].h = (int32_t)h;
    }
    qsort(K, nh, sizeof(ekey), ekey_cmp);
    int64_t ne = 0;
    for (int64_t i = 0; i < nh;) {
        int64_t j = i;
        while (j < nh && K[j].a == K[i].a && K[j].b == K[i].b) ++j;
        if (j - i > 2) { free(K); om_mesh_destroy(m); return -2; }   /* non-manifold edge */
        if (j - i == 2) {
            int32_t h0 = K[i].h, h1 = K[i + 1].h;
            if (F[h0] == F[h1]) { free(K); om_mesh_destroy(m); return -2; }  /* inconsistent orientation */
            m->twin[h0] = h1; m->twin[h1] = h0;
            m->edge[h0] = m->edge[h1] = (int32_t)ne;
        } else {
            m->twin[K[i].h] = -1; m->edge[K[i].h] = (int32_t)ne;
        }
        ++ne; i = j;
    }
    m->ne = ne;
    free(K);

    /* per-face planar layout and 3D frame */
    for (int64_t f = 0; f < nf; ++f) {
        const double* x0 = X + 3 * F[3 * f];
        const double* x1 = X + 3 * F[3 * f + 1];
        const double* x2 = X + 3 * F[3 * f + 2];
        double a[3], b[3];
        for (int c = 0; c < 3; ++c) { a[c] = x1[c] - x0[c]; b[c] = x2[c] - x0[c]; }
        min_image(m, a); min_image(m, b);
        double La = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double e1[3] = {a[0] / La, a[1] / La, a[2] / La};
        double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0)) { om_mesh_destroy(m); return -2; }          /* degenerate face */
        for (int c = 0; c < 3; ++c) n[c] /= nn;
        double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
        m->lay[3 * f] = La;
        m->lay[3 * f + 1] = b[0] * e1[0] + b[1] * e1[1] + b[2] * e1[2];
        m->lay[3 * f + 2] = b[0] * e2[0] + b[1] * e2[1] + b[2] * e2[2];
        for (int c = 0; c < 3; ++c) {
            m->frame[9 * f + c] = x0[c]; m->frame[9 * f + 3 + c] = e1[c]; m->frame[9 * f + 6 + c] = e2[c];
        }
    }
    /* half-edge frames and corner angles */
    for (int64_t h = 0; h < nh; ++h) {
        int64_t f = h / 3; int k = (int)(h % 3);
        double ax, ay, bx, by, cx, cy;
        face_pt(m, f, k, &ax, &ay); face_pt(m, f, k + 1, &bx, &by); face_pt(m, f, k + 2, &cx, &cy);
        double L = hypot(bx - ax, by - ay);
        double dx = (bx - ax) / L, dy = (by - ay) / L;
        m->hl[h] = L;
        m->hcx[h] = dot2(cx - ax, cy - ay, dx, dy);
        m->hcy[h] = cross2(dx, dy, cx - ax, cy - ay);
        /* corner angle at P_k between edges to P_{k+1} and P_{k+2} */
        double ang = atan2(cross2(bx - ax, by - ay, cx - ax, cy - ay), dot2(bx - ax, by - ay, cx - ax, cy - ay));
        m->theta[F[h]] += ang;
        if (m->twin[h] < 0) { m->bnd[F[h]] = 1; m->bnd[F[3 * f + (k + 1) % 3]] = 1; }
    }
    /* pseudo-source vertices: boundary, flat or saddle (angle sum >= 2 pi, 1e-9 slack) */
    for (int64_t v = 0; v < nv; ++v)
        m->pseudo[v] = (uint8_t)(m->bnd[v] || m->theta[v] >= 2.0 * OM_PI - 1e-9);
    /* one-ring corners */
    m->ring_start = (int32_t*)calloc(nv + 1, sizeof(int32_t));
    m->ring = (int32_t*)malloc(sizeof(int32_t) * nh);
    for (int64_t h = 0; h < nh; ++h) m->ring_start[F[h] + 1]++;
    for (int64_t v = 0; v < nv; ++v) m->ring_start[v + 1] += m->ring_start[v];
    int32_t* fill = (int32_t*)calloc(nv, sizeof(int32_t));
    for (int64_t h = 0; h < nh; ++h) m->ring[m->ring_start[F[h]] + fill[F[h]]++] = (int32_t)h;
    free(fill);
    *out = m;
    return 0;
}

void om_mesh_destroy(om_mesh* m) {
    if (!m) return;
    free(m->X); free(m->F); free(m->twin); free(m->edge); free(m->hl); free(m->hcx); free(m->hcy);
    free(m->lay); free(m->frame); free(m->theta); free(m->bnd); free(m->pseudo);
    free(m->ring_start); free(m->ring); free(m);
}

int64_t om_mesh_num_edges(const om_mesh* m) { return m->ne; }

void om_mesh_vertex_info(const om_mesh* m, double* theta, uint8_t* pseudo, uint8_t* boundary) {
    for (int64_t v = 0; v < m->nv; ++v) {
        if (theta) theta[v] = m->theta[v];
        if (pseudo) pseudo[v] = m->pseudo[v];
        if (boundary) boundary[v] = m->bnd[v];
    }
}

void om_face_frame(const om_mesh* m, int32_t f, double* out9) { memcpy(out9, m->frame + 9 * (int64_t)f, 9 * sizeof(double)); }

static void face_to_world_vec(const om_mesh* m, int64_t f, double vx, double vy, double* out3) {
    const double* fr = m->frame + 9 * f;
    for (int c = 0; c < 3; ++c) out3[c] = vx * fr[3 + c] + vy * fr[6 + c];
}
static void world_to_face_vec(const om_mesh* m, int64_t f, const double* v3, double* vx, double* vy) {
    const double* fr = m->frame + 9 * f;
    *vx = v3[0] * fr[3] + v3[1] * fr[4] + v3[2] * fr[5];
    *vy = v3[0] * fr[6] + v3[1] * fr[7] + v3[2] * fr[8];
}
static void bary_to_face(const om_mesh* m, int64_t f, const double* b, double* px, double* py) {
    *px = b[1] * m->lay[3 * f] + b[2] * m->lay[3 * f + 1];
    *py = b[2] * m->lay[3 * f + 2];
}

void om_world_position(const om_mesh* m, int32_t f, const double* bary, double* out3) {
    double px, py, v[3];
    bary_to_face(m, f, bary, &px, &py);
    face_to_world_vec(m, f, px, py, v);
    for (int c = 0; c < 3; ++c) out3[c] = m->frame[9 * (int64_t)f + c] + v[c];
    if (m->periodic)
        for (int a = 0; a < 2; ++a) out3[a] -= m->per[a] * floor(out3[a] / m->per[a]);
}

/* ------------------------------------------------------------------ windows (Sec. 2.2, Sec. 3.1) */
typedef struct {
    int32_t he;          /* half-edge it lies on and propagates into */
    int32_t pv;          /* its pseudo-source vertex, -1 for the source point itself */
    int8_t alive, processed, fixed;
    double b0, b1;       /* interval along the half-edge, 0 <= b0 < b1 <= L */
    double sx, sy;       /* pseudo-source in the half-edge frame, sy <= 0 */
    double sigma;        /* geodesic length from the source to the pseudo-source */
    double ta, tb;       /* fixed==0: image of the source-face x axis; fixed==1: tangent at source */
} owin;

typedef struct { double key; int32_t type; int32_t id; } hent;   /* type 0 window, 1 vertex */

typedef struct {
    const om_mesh* m;
    double rc;
    double* d; double* tv; int32_t* vtouch; int64_t nvt;
    /* how each vertex's distance was reached (path extraction): the previous node of the
       path (a pseudo-source vertex, -1 = the source), a face holding the vertex and its
       corner there, the unit direction from the vertex towards that node in the face's
       layout (it may point into another face of the vertex's ring) and the leg's length */
    int32_t* par; int32_t* pf; int32_t* pc; double* pdir; double* plen;
    int32_t** el; int32_t* ecnt; int32_t* ecap; int32_t* etouch; int64_t net;
    owin* w; int64_t nw, wcap;
    hent* hp; int64_t nh, hcap;
    om_stats st;
} ows;

static ows* ws_create(const om_mesh* m) {
    ows* s = (ows*)calloc(1, sizeof(ows));
    s->m = m;
    s->d = (double*)malloc(sizeof(double) * m->nv);
    for (int64_t v = 0; v < m->nv; ++v) s->d[v] = OM_INF;
    s->tv = (double*)calloc(2 * m->nv, sizeof(double));
    s->vtouch = (int32_t*)malloc(sizeof(int32_t) * m->nv);
    s->par = (int32_t*)malloc(sizeof(int32_t) * m->nv);
    s->pf = (int32_t*)malloc(sizeof(int32_t) * m->nv);
    s->pc = (int32_t*)malloc(sizeof(int32_t) * m->nv);
    s->pdir = (double*)malloc(sizeof(double) * 2 * m->nv);
    s->plen = (double*)malloc(sizeof(double) * m->nv);
    s->el = (int32_t**)calloc(m->ne, sizeof(int32_t*));
    s->ecnt = (int32_t*)calloc(m->ne, sizeof(int32_t));
    s->ecap = (int32_t*)calloc(m->ne, sizeof(int32_t));
    s->etouch = (int32_t*)malloc(sizeof(int32_t) * m->ne);
    s->wcap = 1024; s->w = (owin*)malloc(sizeof(owin) * s->wcap);
    s->hcap = 1024; s->hp = (hent*)malloc(sizeof(hent) * s->hcap);
    return s;
}

static void ws_reset(ows* s) {
    for (int64_t i = 0; i < s->nvt; ++i) s->d[s->vtouch[i]] = OM_INF;
    for (int64_t i = 0; i < s->net; ++i) s->ecnt[s->etouch[i]] = 0;
    s->nvt = 0; s->net = 0; s->nw = 0; s->nh = 0;
}

static void ws_destroy(ows* s) {
    for (int64_t e = 0; e < s->m->ne; ++e) free(s->el[e]);
    free(s->d); free(s->tv); free(s->vtouch);
    free(s->par); free(s->pf); free(s->pc); free(s->pdir); free(s->plen); free(s->el); free(s->ecnt); free(s->ecap);
    free(s->etouch); free(s->w); free(s->hp); free(s);
}

static void heap_push(ows* s, double key, int32_t type, int32_t id) {
    if (s->nh == s->hcap) { s->hcap *= 2; s->hp = (hent*)realloc(s->hp, sizeof(hent) * s->hcap); }
    int64_t i = s->nh++;
    hent e = {key, type, id};
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (s->hp[p].key <= key) break;
        s->hp[i] = s->hp[p]; i = p;
    }
    s->hp[i] = e;
}

static hent heap_pop(ows* s) {
    hent top = s->hp[0];
    hent last = s->hp[--s->nh];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= s->nh) break;
        if (c + 1 < s->nh && s->hp[c + 1].key < s->hp[c].key) ++c;
        if (s->hp[c].key >= last.key) break;
        s->hp[i] = s->hp[c]; i = c;
    }
    if (s->nh > 0) s->hp[i] = last;
    return top;
}

/* smallest distance the window carries over its interval */
static double win_key(const owin* w) {
    double x = w->sx < w->b0 ? w->b0 : (w->sx > w->b1 ? w->b1 : w->sx);
    return w->sigma + hypot(x - w->sx, w->sy);
}

/* initial direction at the source (in the source face layout) of the path the window
 * carries to the point (px, py) of its half-edge frame */
static void win_tangent(const owin* w, double px, double py, double* tx, double* ty) {
    if (w->fixed) { *tx = w->ta; *ty = w->tb; return; }
    double dx = px - w->sx, dy = py - w->sy, n = hypot(dx, dy);
    dx /= n; dy /= n;
    *tx = dx * w->ta + dy * w->tb;
    *ty = -dx * w->tb + dy * w->ta;
}

/* A pseudo-source on the edge line (|s.y| ~ 0) sees the face beyond it only through its
 * own position: the whole face when s lies inside [b0, b1], nothing otherwise. */
static int win_degenerate(const om_mesh* m, const owin* w) { return w->sy > -1e-13 * m->hl[w->he]; }
static int win_degenerate_sees(const om_mesh* m, const owin* w) {
    const double tol = 1e-12 * m->hl[w->he];
    return w->sx >= w->b0 - tol && w->sx <= w->b1 + tol;
}

/* previous node of a path, as recorded for the path extraction */
typedef struct { int32_t par, f, k; double dx, dy, len; } olink;

static void set_link(ows* s, int32_t v, const olink* l) {
    s->par[v] = l->par; s->pf[v] = l->f; s->pc[v] = l->k;
    s->pdir[2 * v] = l->dx; s->pdir[2 * v + 1] = l->dy; s->plen[v] = l->len;
}

static void set_vertex(ows* s, int32_t v, double dist, double tx, double ty, const olink* l) {
    if (!(dist < s->d[v])) {
        /* an equally short path (up to rounding) that comes straight from the source is
           preferred as the vertex's previous node: distances and tangents do not change */
        if (dist <= s->d[v] * (1.0 + 1e-13) && l->par < 0 && s->par[v] >= 0) set_link(s, v, l);
        return;
    }
    if (s->d[v] == OM_INF) s->vtouch[s->nvt++] = v;
    s->d[v] = dist;
    s->tv[2 * v] = tx; s->tv[2 * v + 1] = ty;
    set_link(s, v, l);
    if (s->m->pseudo[v] && dist < s->rc) heap_push(s, dist, 1, v);
}

/* vector (a, b) of the frame of half-edge 3f+k -> face f's layout */
static void he_vec_to_layout(const om_mesh* m, int64_t f, int k, double a, double b, double* x, double* y) {
    double ax, ay, bx, by;
    face_pt(m, f, k, &ax, &ay);
    face_pt(m, f, k + 1, &bx, &by);
    const double L = hypot(bx - ax, by - ay);
    const double dx = (bx - ax) / L, dy = (by - ay) / L;
    *x = a * dx - b * dy;
    *y = a * dy + b * dx;
}

/* the link of a point (X, Y) of window W's half-edge frame straight back to W's
   pseudo-source.  which = 2: the far corner of the face W enters (the direction lies in
   that face); 0 / 1: the start / end vertex of W's edge (the direction points into the
   face on the other side of the edge, and is written in that face); -1: a point inside
   the face W enters. */
static void window_link(const om_mesh* m, const owin* W, double X, double Y, int which, olink* l) {
    const int64_t f = W->he / 3; const int k = W->he % 3;
    const double a = W->sx - X, b = W->sy - Y, n = hypot(a, b);
    l->par = W->pv; l->len = n;
    const double ua = n > 0.0 ? a / n : 1.0, ub = n > 0.0 ? b / n : 0.0;
    if (which == 0 || which == 1) {
        const int32_t tw = m->twin[W->he];
        const int64_t g = tw / 3; const int kg = tw % 3;   /* tw runs from W's end vertex to its start */
        l->f = (int32_t)g; l->k = which == 0 ? (kg + 1) % 3 : kg;
        he_vec_to_layout(m, g, kg, -ua, -ub, &l->dx, &l->dy);
    } else {
        l->f = (int32_t)f; l->k = which == 2 ? (k + 2) % 3 : -1;
        he_vec_to_layout(m, f, k, ua, ub, &l->dx, &l->dy);
    }
}

static int32_t new_window(ows* s, const owin* w) {
    if (s->nw == s->wcap) { s->wcap *= 2; s->w = (owin*)realloc(s->w, sizeof(owin) * s->wcap); }
    s->w[s->nw] = *w;
    return (int32_t)s->nw++;
}

static void edge_append(ows* s, int32_t e, int32_t id) {
    if (s->ecnt[e] == 0) s->etouch[s->net++] = e;
    if (s->ecnt[e] == s->ecap[e]) {
        s->ecap[e] = s->ecap[e] ? 2 * s->ecap[e] : 4;
        s->el[e] = (int32_t*)realloc(s->el[e], sizeof(int32_t) * s->ecap[e]);
    }
    s->el[e][s->ecnt[e]++] = id;
}

/* D(x) = (sa + |x - a|) - (sb + |x - b|) for a point (x, 0) */
static double dist_diff(double x, double ax, double ay, double sa, double bx, double by, double sb) {
    return (sa + hypot(x - ax, ay)) - (sb + hypot(x - bx, by));
}

/* Points x in (lo, hi) where the two distance functions of windows a and b are equal:
 * |x-a| - |x-b| = sb - sa, squared twice into a quadratic; spurious roots only add
 * breakpoints because the caller decides the winner of every piece by evaluation. */
static int equal_dist_points(double ax, double ay, double sa, double bx, double by, double sb,
                             double lo, double hi, double* r) {
    double del = sb - sa;
    double al = bx - ax;
    double be = (ax * ax + ay * ay) - (bx * bx + by * by) - del * del;
    double c2 = del * del - al * al;
    double c1 = -(2.0 * del * del * bx + al * be);
    double c0 = del * del * (bx * bx + by * by) - 0.25 * be * be;
    double cand[2]; int nc = 0;
    double scale = fabs(c2) + fabs(c1) / (fabs(hi) + fabs(lo) + 1e-300) + 1e-300;
    if (fabs(c2) <= 1e-14 * scale) {
        if (c1 != 0.0) cand[nc++] = -c0 / c1;
    } else {
        double disc = c1 * c1 - 4.0 * c2 * c0;
        if (disc < 0.0) disc = 0.0;   /* tangency: no sign change, a breakpoint is harmless */
        double sq = sqrt(disc);
        double q = -0.5 * (c1 + (c1 >= 0.0 ? sq : -sq));
        if (q != 0.0) { cand[nc++] = q / c2; cand[nc++] = c0 / q; }
        else cand[nc++] = -c1 / (2.0 * c2);
    }
    int n = 0;
    for (int i = 0; i < nc; ++i)
        if (cand[i] > lo && cand[i] < hi) r[n++] = cand[i];
    if (n == 2 && r[0] > r[1]) { double t = r[0]; r[0] = r[1]; r[1] = t; }
    return n;
}

#define OM_MAXP 64

/* append [x0, x1] to an interval list, merging with a touching last interval */
static void ivl_add(double (*iv)[2], int* n, double x0, double x1) {
    if (x1 <= x0) return;
    if (*n > 0 && x0 <= iv[*n - 1][1]) { if (x1 > iv[*n - 1][1]) iv[*n - 1][1] = x1; return; }
    if (*n < OM_MAXP) { iv[*n][0] = x0; iv[*n][1] = x1; ++*n; }
}

/* Insert a candidate window on its edge, intersecting it with every window already on
 * that edge (from either side): on every overlap each keeps only the part where it
 * carries the smaller distance (ties go to the window already there). */
static void insert_window(ows* s, owin cand) {
    const om_mesh* m = s->m;
    const int32_t h = cand.he;
    const double L = m->hl[h];
    const double tolw = 1e-12 * L;
    if (cand.b0 < 0.0) cand.b0 = 0.0;
    if (cand.b1 > L) cand.b1 = L;
    if (cand.b1 - cand.b0 <= tolw || win_key(&cand) >= s->rc) { s->st.windows_dropped++; return; }
    double pc[OM_MAXP][2]; int np = 1;
    pc[0][0] = cand.b0; pc[0][1] = cand.b1;
    const int32_t e = m->edge[h];
    const int32_t n_exist = s->ecnt[e];
    for (int32_t i = 0; i < n_exist && np > 0; ++i) {
        int32_t oid = s->el[e][i];
        owin* o = &s->w[oid];
        if (!o->alive) continue;
        const int same = (o->he == h);
        double o0 = same ? o->b0 : L - o->b1, o1 = same ? o->b1 : L - o->b0;
        double osx = same ? o->sx : L - o->sx, osy = same ? o->sy : -o->sy;
        double npc[OM_MAXP][2]; int nn = 0;
        double lost[OM_MAXP][2]; int nl = 0;
        for (int p = 0; p < np; ++p) {
            double a0 = pc[p][0], a1 = pc[p][1];
            double lo = a0 > o0 ? a0 : o0, hi = a1 < o1 ? a1 : o1;
            if (hi - lo <= tolw) { ivl_add(npc, &nn, a0, a1); continue; }
            double bp[4]; int nb = 0;
            bp[nb++] = lo;
            double r[2];
            int nr = equal_dist_points(cand.sx, cand.sy, cand.sigma, osx, osy, o->sigma, lo, hi, r);
            for (int q = 0; q < nr; ++q) bp[nb++] = r[q];
            bp[nb++] = hi;
            ivl_add(npc, &nn, a0, lo);
            for (int q = 0; q + 1 < nb; ++q) {
                double x0 = bp[q], x1 = bp[q + 1];
                double xm = 0.5 * (x0 + x1);
                double dd = dist_diff(xm, cand.sx, cand.sy, cand.sigma, osx, osy, o->sigma);
                if (dd < 0.0) { ivl_add(npc, &nn, x0, x1); ivl_add(lost, &nl, x0, x1); }
            }
            ivl_add(npc, &nn, hi, a1);
        }
        np = 0;
        for (int p = 0; p < nn; ++p)
            if (npc[p][1] - npc[p][0] > tolw) { pc[np][0] = npc[p][0]; pc[np][1] = npc[p][1]; ++np; }
        if (nl > 0) {
            /* o keeps [o0, o1] minus the lost intervals (candidate frame) */
            double keep[OM_MAXP][2]; int nk = 0;
            double cur = o0;
            for (int q = 0; q < nl; ++q) {
                if (lost[q][0] - cur > tolw) ivl_add(keep, &nk, cur, lost[q][0]);
                if (lost[q][1] > cur) cur = lost[q][1];
            }
            if (o1 - cur > tolw) ivl_add(keep, &nk, cur, o1);
            owin base = *o;
            if (nk == 0) { o->alive = 0; continue; }
            for (int q = 0; q < nk; ++q) {
                double k0 = same ? keep[q][0] : L - keep[q][1];
                double k1 = same ? keep[q][1] : L - keep[q][0];
                if (q == 0) { s->w[oid].b0 = k0; s->w[oid].b1 = k1; }
                else {
                    owin piece = base; piece.b0 = k0; piece.b1 = k1;
                    int32_t pid = new_window(s, &piece);
                    edge_append(s, e, pid);
                    s->st.windows_created++;
                    if (!piece.processed) heap_push(s, win_key(&piece), 0, pid);
                }
            }
        }
    }
    if (np == 0) { s->st.windows_dropped++; return; }
    for (int p = 0; p < np; ++p) {
        owin w = cand;
        w.b0 = pc[p][0]; w.b1 = pc[p][1];
        w.alive = 1; w.processed = 0;
        double key = win_key(&w);
        if (key >= s->rc) continue;
        int32_t id = new_window(s, &w);
        edge_append(s, e, id);
        s->st.windows_created++;
        heap_push(s, key, 0, id);
    }
}

/* parameter mu in [0,1] along A->B where the ray from s through (X, 0) meets line AB */
static double ray_hit(double sx, double sy, double X, double ax, double ay, double bx, double by) {
    double dx = X - sx, dy = -sy;
    double den = cross2(bx - ax, by - ay, dx, dy);
    double mu = den != 0.0 ? cross2(sx - ax, sy - ay, dx, dy) / den : 0.0;
    return mu < 0.0 ? 0.0 : (mu > 1.0 ? 1.0 : mu);
}

/* Unfold window w across its half-edge into the next face (Sec. 2.2 / Sec. 3.1):
 * the opposite vertex c is placed in the window frame, the cone from s through
 * [b0, b1] is cut by the two far edges into at most two child windows, and the
 * vertices reached directly receive distance candidates. */
static void propagate(ows* s, int32_t wid) {
    const om_mesh* m = s->m;
    s->w[wid].processed = 1;
    const owin W = s->w[wid];
    s->st.windows_propagated++;
    const int32_t h = W.he;
    const int64_t f = h / 3; const int k = h % 3;
    const double L = m->hl[h], cx = m->hcx[h], cy = m->hcy[h];
    const int32_t vu = m->F[3 * f + k], vv = m->F[3 * f + (k + 1) % 3], vc = m->F[3 * f + (k + 2) % 3];
    const double tolv = 1e-12 * L;
    double tx, ty;
    olink lk;
    if (W.b0 <= tolv) {
        win_tangent(&W, 0.0, 0.0, &tx, &ty);
        window_link(m, &W, 0.0, 0.0, 0, &lk);
        set_vertex(s, vu, W.sigma + hypot(W.sx, W.sy), tx, ty, &lk);
    }
    if (W.b1 >= L - tolv) {
        win_tangent(&W, L, 0.0, &tx, &ty);
        window_link(m, &W, L, 0.0, 1, &lk);
        set_vertex(s, vv, W.sigma + hypot(L - W.sx, W.sy), tx, ty, &lk);
    }
    const int degen = win_degenerate(m, &W);
    if (degen && !win_degenerate_sees(m, &W)) return;
    const double xc = degen ? 0.5 * (W.b0 + W.b1) : W.sx + (cx - W.sx) * (-W.sy) / (cy - W.sy);
    if (degen || (xc >= W.b0 && xc <= W.b1)) {
        win_tangent(&W, cx, cy, &tx, &ty);
        window_link(m, &W, cx, cy, 2, &lk);
        set_vertex(s, vc, W.sigma + hypot(cx - W.sx, cy - W.sy), tx, ty, &lk);
    }
    const int32_t tl = m->twin[3 * f + (k + 2) % 3];   /* across edge c-u */
    const int32_t tr = m->twin[3 * f + (k + 1) % 3];   /* across edge v-c */
    const double Lc = hypot(cx, cy), Ld = hypot(L - cx, cy);
    if (tl >= 0 && (degen || xc > W.b0)) {
        double mu0 = 0.0, mu1 = 1.0;
        if (!degen) {
            mu0 = ray_hit(W.sx, W.sy, W.b0, 0.0, 0.0, cx, cy);
            mu1 = (W.b1 >= xc) ? 1.0 : ray_hit(W.sx, W.sy, W.b1, 0.0, 0.0, cx, cy);
        }
        const double co = cx / Lc, si = cy / Lc;     /* rotate by -angle(c), origin u */
        owin c = W;
        c.he = tl;
        c.sx = W.sx * co + W.sy * si;
        c.sy = -W.sx * si + W.sy * co;
        if (!W.fixed) { c.ta = W.ta * co + W.tb * si; c.tb = -W.ta * si + W.tb * co; }
        const double Lt = m->hl[tl];
        c.b0 = mu0 * Lt; c.b1 = mu1 * Lt;
        if (c.sy > 0.0) c.sy = 0.0;
        insert_window(s, c);
    }
    if (tr >= 0 && (degen || xc < W.b1)) {
        double mu0 = 0.0, mu1 = 1.0;
        if (!degen) {
            mu0 = (W.b0 <= xc) ? 0.0 : ray_hit(W.sx, W.sy, W.b0, cx, cy, L, 0.0);
            mu1 = ray_hit(W.sx, W.sy, W.b1, cx, cy, L, 0.0);
        }
        const double co = (L - cx) / Ld, si = -cy / Ld;   /* rotate by -angle(v - c), origin c */
        owin c = W;
        c.he = tr;
        const double px = W.sx - cx, py = W.sy - cy;
        c.sx = px * co + py * si;
        c.sy = -px * si + py * co;
        if (!W.fixed) { c.ta = W.ta * co + W.tb * si; c.tb = -W.ta * si + W.tb * co; }
        const double Lt = m->hl[tr];
        c.b0 = mu0 * Lt; c.b1 = mu1 * Lt;
        if (c.sy > 0.0) c.sy = 0.0;
        insert_window(s, c);
    }
}

/* A boundary, flat or saddle vertex reached at distance d(v) acts as a new pseudo-source:
 * shortest paths may bend there, so it starts a window on every edge opposite to it. */
static void emit_vertex(ows* s, int32_t v) {
    const om_mesh* m = s->m;
    s->st.vertex_events++;
    for (int32_t r = m->ring_start[v]; r < m->ring_start[v + 1]; ++r) {
        const int32_t hc = m->ring[r];
        const int64_t f = hc / 3; const int k = hc % 3;
        const int32_t hop = (int32_t)(3 * f + (k + 1) % 3);
        const int32_t tw = m->twin[hop];
        if (tw < 0) continue;
        const double L = m->hl[hop];
        owin c;
        memset(&c, 0, sizeof(c));
        c.he = tw; c.b0 = 0.0; c.b1 = m->hl[tw];
        c.sx = L - m->hcx[hop]; c.sy = -m->hcy[hop];
        c.sigma = s->d[v]; c.fixed = 1; c.pv = v;
        c.ta = s->tv[2 * v]; c.tb = s->tv[2 * v + 1];
        insert_window(s, c);
    }
}

/* Build the window structure of one source point (face f0, barycentrics b). */
static void run_source(ows* s, int32_t f0, const double* b) {
    const om_mesh* m = s->m;
    ws_reset(s);
    s->st.sources++;
    double qx, qy;
    bary_to_face(m, f0, b, &qx, &qy);
    for (int k = 0; k < 3; ++k) {
        double px, py;
        face_pt(m, f0, k, &px, &py);
        double dd = hypot(px - qx, py - qy);
        double tx = dd > 0.0 ? (px - qx) / dd : 1.0, ty = dd > 0.0 ? (py - qy) / dd : 0.0;
        const olink lk = {-1, f0, k, -tx, -ty, dd};
        set_vertex(s, m->F[3 * f0 + k], dd, tx, ty, &lk);
    }
    for (int k = 0; k < 3; ++k) {
        const int32_t h = 3 * f0 + k, tw = m->twin[h];
        if (tw < 0) continue;
        double ax, ay, bx, by;
        face_pt(m, f0, k, &ax, &ay); face_pt(m, f0, k + 1, &bx, &by);
        const double L = m->hl[h];
        const double dx = (bx - ax) / L, dy = (by - ay) / L;
        const double hx = dot2(qx - ax, qy - ay, dx, dy), hy = cross2(dx, dy, qx - ax, qy - ay);
        owin c;
        memset(&c, 0, sizeof(c));
        c.he = tw; c.b0 = 0.0; c.b1 = m->hl[tw];
        c.sx = L - hx; c.sy = -hy; if (c.sy > 0.0) c.sy = 0.0;
        c.sigma = 0.0; c.fixed = 0; c.pv = -1;
        c.ta = -dx; c.tb = dy;
        insert_window(s, c);
    }
    while (s->nh > 0) {
        hent e = heap_pop(s);
        if (e.key >= s->rc) break;
        if (e.type == 1) {
            if (e.key > s->d[e.id]) continue;     /* superseded by a shorter distance */
            emit_vertex(s, e.id);
        } else {
            owin* w = &s->w[e.id];
            if (!w->alive || w->processed) continue;
            double key = win_key(w);
            if (key > e.key) { if (key < s->rc) heap_push(s, key, 0, e.id); continue; }
            propagate(s, e.id);
        }
    }
}

/* candidate (length, tangent) list of one query, to report how far the runner-up with a
 * different tangent is (a near-tie marks a cut-locus point where the tangent is set-valued) */
#define OM_MAXCAND 64
typedef struct { int n; double d[OM_MAXCAND], tx[OM_MAXCAND], ty[OM_MAXCAND]; } ocand;
static void cand_add(ocand* c, double d, double tx, double ty) {
    if (c && c->n < OM_MAXCAND) { c->d[c->n] = d; c->tx[c->n] = tx; c->ty[c->n] = ty; c->n++; }
}
static double cand_gap(const ocand* c, double best, double tx, double ty) {
    double g = OM_INF;
    for (int i = 0; i < c->n; ++i)
        if (hypot(c->tx[i] - tx, c->ty[i] - ty) > 1e-9 && c->d[i] - best < g) g = c->d[i] - best;
    return g;
}

/* Distance and source tangent (source-face layout) of a target point: the minimum over
 * the direct segment (same face), windows entering the face whose cone contains the
 * point, and paths through the face's vertices (Sec. 3.1: query the cached structure). */
static double query_point_c(ows* s, int32_t f0, double qx, double qy, int32_t f, const double* b,
                            double* tx, double* ty, ocand* cands, olink* lk) {
    const om_mesh* m = s->m;
    s->st.queries++;
    double px, py;
    bary_to_face(m, f, b, &px, &py);
    double best = OM_INF; *tx = 0.0; *ty = 0.0;
    olink lb = {-1, f, -1, 1.0, 0.0, 0.0};
    if (f == f0) {
        best = hypot(px - qx, py - qy);
        if (best > 0.0) { *tx = (px - qx) / best; *ty = (py - qy) / best; }
        cand_add(cands, best, *tx, *ty);
        lb.dx = best > 0.0 ? -*tx : 1.0; lb.dy = best > 0.0 ? -*ty : 0.0; lb.len = best;
    }
    for (int k = 0; k < 3; ++k) {
        const int32_t h = 3 * f + k, e = m->edge[h];
        double hx = 0.0, hy = 0.0; int have = 0;
        for (int32_t i = 0; i < s->ecnt[e]; ++i) {
            const owin* w = &s->w[s->el[e][i]];
            if (!w->alive || w->he != h) continue;
            if (!have) { to_he_frame(m, f, k, px, py, &hx, &hy); have = 1; }
            int inside;
            if (win_degenerate(m, w)) inside = win_degenerate_sees(m, w);
            else {
                const double X = w->sx + (hx - w->sx) * (-w->sy) / (hy - w->sy);
                const double tol = 1e-12 * m->hl[h];
                inside = (X >= w->b0 - tol && X <= w->b1 + tol);
            }
            if (!inside) continue;
            const double dd = w->sigma + hypot(hx - w->sx, hy - w->sy);
            double ux, uy;
            win_tangent(w, hx, hy, &ux, &uy);
            cand_add(cands, dd, ux, uy);
            if (dd < best) {
                best = dd; *tx = ux; *ty = uy;
                window_link(m, w, hx, hy, -1, &lb);
                lb.f = f;
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        const int32_t v = m->F[3 * f + k];
        if (s->d[v] == OM_INF) continue;
        double vx, vy;
        face_pt(m, f, k, &vx, &vy);
        const double dd = s->d[v] + hypot(px - vx, py - vy);
        cand_add(cands, dd, s->tv[2 * v], s->tv[2 * v + 1]);
        if (dd < best) {
            best = dd; *tx = s->tv[2 * v]; *ty = s->tv[2 * v + 1];
            const double n = hypot(vx - px, vy - py);
            lb.par = v; lb.f = f; lb.k = -1; lb.len = n;
            lb.dx = n > 0.0 ? (vx - px) / n : 1.0; lb.dy = n > 0.0 ? (vy - py) / n : 0.0;
        }
    }
    if (lk) *lk = lb;
    return best;
}

static double query_point(ows* s, int32_t f0, double qx, double qy, int32_t f, const double* b,
                          double* tx, double* ty) {
    return query_point_c(s, f0, qx, qy, f, b, tx, ty, NULL, NULL);
}

static void add_stats(om_stats* a, const om_stats* b) {
    a->windows_created += b->windows_created; a->windows_propagated += b->windows_propagated;
    a->windows_dropped += b->windows_dropped; a->vertex_events += b->vertex_events;
    a->sources += b->sources; a->queries += b->queries;
}

int om_geodesic_query(const om_mesh* m, int32_t f0, const double* bary0, double r_c,
                      int64_t nt, const int32_t* tf, const double* tb,
                      double* dist, double* tan3, om_stats* st) {
    if (f0 < 0 || f0 >= m->nf) return -1;
    ows* s = ws_create(m);
    s->rc = r_c;
    run_source(s, f0, bary0);
    double qx, qy;
    bary_to_face(m, f0, bary0, &qx, &qy);
    for (int64_t t = 0; t < nt; ++t) {
        double tx, ty;
        double d = query_point(s, f0, qx, qy, tf[t], tb + 3 * t, &tx, &ty);
        if (!(d < r_c)) { dist[t] = OM_INF; tan3[3 * t] = tan3[3 * t + 1] = tan3[3 * t + 2] = 0.0; }
        else { dist[t] = d; face_to_world_vec(m, f0, tx, ty, tan3 + 3 * t); }
    }
    if (st) add_stats(st, &s->st);
    ws_destroy(s);
    return 0;
}

/* ------------------------------------------------------------------ neighbour lists (Sec. 3.1) */
/* Euclidean distance (minimum image on periodic meshes): a lower bound of the geodesic one */
static double euclid(const om_mesh* m, const double* a, const double* b) {
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    min_image(m, d);
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

typedef struct { int32_t j; double d, t[3], gap; } opair;

static int cmp_pair(const void* a, const void* b) {
    const opair* x = (const opair*)a; const opair* y = (const opair*)b;
    return (x->j > y->j) - (x->j < y->j);
}

int om_neighbors_subset(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
                        double r_c, int64_t ns, const int64_t* src, int64_t cap,
                        int64_t* n_pairs, int64_t* row_start, int32_t* nbr_j, double* dist,
                        double* tan3, int nthreads, om_stats* st) {
    return om_neighbors_gap(m, n, face, bary, r_c, ns, src, cap, n_pairs, row_start, nbr_j, dist, tan3,
                            NULL, nthreads, st);
}

int om_neighbors_gap(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
                     double r_c, int64_t ns, const int64_t* src, int64_t cap,
                     int64_t* n_pairs, int64_t* row_start, int32_t* nbr_j, double* dist,
                     double* tan3, double* gap, int nthreads, om_stats* st) {
    for (int64_t i = 0; i < n; ++i) if (face[i] < 0 || face[i] >= m->nf) return -1;
    double* x = (double*)malloc(sizeof(double) * 3 * n);
    for (int64_t i = 0; i < n; ++i) om_world_position(m, face[i], bary + 3 * i, x + 3 * i);
    opair** rows = (opair**)calloc(ns, sizeof(opair*));
    int64_t* cnt = (int64_t*)calloc(ns, sizeof(int64_t));
    om_stats tot; memset(&tot, 0, sizeof(tot));
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        ows* s = ws_create(m);
        s->rc = r_c;
        opair* buf = (opair*)malloc(sizeof(opair) * (n > 0 ? n : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t r = 0; r < ns; ++r) {
            const int64_t i = src[r];
            run_source(s, face[i], bary + 3 * i);
            double qx, qy;
            bary_to_face(m, face[i], bary + 3 * i, &qx, &qy);
            int64_t c = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i || !(euclid(m, x + 3 * i, x + 3 * j) < r_c)) continue;
                double tx, ty;
                ocand cands;
                cands.n = 0;
                double d = query_point_c(s, face[i], qx, qy, face[j], bary + 3 * j, &tx, &ty, &cands, NULL);
                if (!(d < r_c)) continue;
                buf[c].j = (int32_t)j; buf[c].d = d;
                buf[c].gap = cand_gap(&cands, d, tx, ty);
                face_to_world_vec(m, face[i], tx, ty, buf[c].t);
                ++c;
            }
            rows[r] = (opair*)malloc(sizeof(opair) * (c > 0 ? c : 1));
            memcpy(rows[r], buf, sizeof(opair) * c);
            cnt[r] = c;
        }
        free(buf);
#ifdef _OPENMP
#pragma omp critical
#endif
        add_stats(&tot, &s->st);
        ws_destroy(s);
    }
    int64_t total = 0;
    for (int64_t r = 0; r < ns; ++r) { row_start[r] = total; total += cnt[r]; }
    row_start[ns] = total;
    *n_pairs = total;
    int rc = 0;
    if (total > cap) rc = -5;
    else {
        for (int64_t r = 0; r < ns; ++r) {
            qsort(rows[r], cnt[r], sizeof(opair), cmp_pair);
            for (int64_t c = 0; c < cnt[r]; ++c) {
                const int64_t o = row_start[r] + c;
                nbr_j[o] = rows[r][c].j; dist[o] = rows[r][c].d;
                if (tan3) for (int a = 0; a < 3; ++a) tan3[3 * o + a] = rows[r][c].t[a];
                if (gap) gap[o] = rows[r][c].gap;
            }
        }
    }
    for (int64_t r = 0; r < ns; ++r) free(rows[r]);
    free(rows); free(cnt); free(x);
    if (st) add_stats(st, &tot);
    return rc;
}

int om_neighbors(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
                 double r_c, int64_t cap, int64_t* n_pairs, int64_t* row_start,
                 int32_t* nbr_j, double* dist, double* tan3, int nthreads, om_stats* st) {
    int64_t* src = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) src[i] = i;
    int rc = om_neighbors_subset(m, n, face, bary, r_c, n, src, cap, n_pairs, row_start,
                                 nbr_j, dist, tan3, nthreads, st);
    free(src);
    return rc;
}

/* ------------------------------------------------------------------ forces (Sec. 2.1, Sec. 3.1) */
double om_pair_energy(const om_potential* p, double l) {
    if (!(l < p->r_cut)) return 0.0;
    if (p->kind == 0) { double u = 1.0 - l / p->sigma; return p->eps * u * u; }
    if (p->kind == 1) { double q = pow(p->sigma / l, 6.0); return 4.0 * p->eps * (q * q - q) + p->eps; }
    return p->A * exp(-l * l / (2.0 * p->sigma * p->sigma));
}

double om_pair_dudl(const om_potential* p, double l) {
    if (!(l < p->r_cut)) return 0.0;
    if (p->kind == 0) return -2.0 * p->eps * (1.0 - l / p->sigma) / p->sigma;
    if (p->kind == 1) { double q = pow(p->sigma / l, 6.0); return 24.0 * p->eps * (q - 2.0 * q * q) / l; }
    return -(l / (p->sigma * p->sigma)) * p->A * exp(-l * l / (2.0 * p->sigma * p->sigma));
}

/* F_i = sum_j -U'(l_ij) grad_{x_i} l_ij with grad_{x_i} l_ij = -(unit initial tangent of the
 * geodesic from i to j), i.e. F_i = sum_j U'(l_ij) t_ij: repulsive for U' < 0. */
int om_forces_subset(const om_mesh* m, int64_t n, const int32_t* face, const double* bary, double r_c,
                     const om_potential* pot, int64_t ns, const int64_t* src, double* F, double* e_src,
                     int nthreads) {
    for (int64_t i = 0; i < n; ++i) if (face[i] < 0 || face[i] >= m->nf) return -1;
    for (int64_t k = 0; src && k < ns; ++k) if (src[k] < 0 || src[k] >= n) return -1;
    double* x = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) om_world_position(m, face[i], bary + 3 * i, x + 3 * i);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        ows* s = ws_create(m);
        s->rc = r_c;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t k = 0; k < ns; ++k) {
            const int64_t i = src ? src[k] : k;
            run_source(s, face[i], bary + 3 * i);
            double qx, qy;
            bary_to_face(m, face[i], bary + 3 * i, &qx, &qy);
            double fx = 0.0, fy = 0.0, e = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i || !(euclid(m, x + 3 * i, x + 3 * j) < r_c)) continue;
                double tx, ty;
                const double d = query_point(s, face[i], qx, qy, face[j], bary + 3 * j, &tx, &ty);
                if (!(d < r_c)) continue;
                const double du = om_pair_dudl(pot, d);
                fx += du * tx; fy += du * ty;
                e += 0.5 * om_pair_energy(pot, d);
            }
            face_to_world_vec(m, face[i], fx, fy, F + 3 * k);
            if (e_src) e_src[k] = e;
        }
        ws_destroy(s);
    }
    free(x);
    return 0;
}

int om_forces(const om_mesh* m, int64_t n, const int32_t* face, const double* bary,
              double r_c, const om_potential* pot, double* F, double* epot, int nthreads) {
    double* e = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    const int rc = om_forces_subset(m, n, face, bary, r_c, pot, n, NULL, F, e, nthreads);
    if (rc == 0 && epot) {
        double sum = 0.0;
        for (int64_t i = 0; i < n; ++i) sum += e[i];
        *epot = sum;
    }
    free(e);
    return rc;
}

/* ------------------------------------------------------------------ face walk (Sec. 3.2) */
static void bary_of(const om_mesh* m, int64_t f, double px, double py, double* l) {
    const double L01 = m->lay[3 * f], x2 = m->lay[3 * f + 1], y2 = m->lay[3 * f + 2];
    l[2] = py / y2;
    l[1] = (px - l[2] * x2) / L01;
    l[0] = 1.0 - l[1] - l[2];
}

static void rot2(double co, double si, double* x, double* y) {
    double a = co * *x - si * *y, b = si * *x + co * *y;
    *x = a; *y = b;
}

#define OM_MAXCARRY 4

/* Straightest continuation through an interior vertex (Polthier-Schmies, as adopted in
 * Sec. 3.2): leave at half the vertex's total angle from the incoming direction.  At a
 * boundary vertex the walk turns back along its incoming direction. */
static void vertex_turn(const om_mesh* m, int64_t* fp, int cw, double* px, double* py,
                        double* dx, double* dy, int nc, double* cx, double* cy) {
    int64_t f = *fp;
    const int32_t v = m->F[3 * f + cw];
    const double len = hypot(*dx, *dy);
    const double ux = *dx / len, uy = *dy / len;
    double phi[OM_MAXCARRY], mag[OM_MAXCARRY];
    for (int i = 0; i < nc; ++i) {
        mag[i] = hypot(cx[i], cy[i]);
        phi[i] = atan2(cross2(ux, uy, cx[i], cy[i]), dot2(ux, uy, cx[i], cy[i]));
    }
    double wx, wy;
    face_pt(m, f, cw, &wx, &wy);
    if (m->bnd[v]) {
        *px = wx; *py = wy; *dx = -*dx; *dy = -*dy;
        for (int i = 0; i < nc; ++i) { cx[i] = -cx[i]; cy[i] = -cy[i]; }
        return;
    }
    double nx, ny;
    face_pt(m, f, cw + 1, &nx, &ny);
    double ex = nx - wx, ey = ny - wy, el = hypot(ex, ey);
    ex /= el; ey /= el;
    /* reversed incoming direction, angle measured counter-clockwise from edge w->P_{cw+1} */
    double beta = atan2(cross2(ex, ey, -ux, -uy), dot2(ex, ey, -ux, -uy));
    if (beta < 0.0) beta = 0.0;
    double rem = beta + 0.5 * m->theta[v];
    for (int guard = 0; guard < 64; ++guard) {
        const int32_t hc = (int32_t)(3 * f + cw);
        double ang = atan2(m->hcy[hc], m->hcx[hc]);   /* corner angle at w in face f */
        if (rem <= ang) break;
        rem -= ang;
        const int32_t hop = (int32_t)(3 * f + (cw + 2) % 3);  /* edge P_{cw+2} -> w */
        const int32_t tw = m->twin[hop];
        if (tw < 0) break;
        f = tw / 3; cw = tw % 3;
    }
    face_pt(m, f, cw, &wx, &wy);
    face_pt(m, f, cw + 1, &nx, &ny);
    ex = nx - wx; ey = ny - wy; el = hypot(ex, ey);
    ex /= el; ey /= el;
    double ox = ex, oy = ey;
    rot2(cos(rem), sin(rem), &ox, &oy);
    *fp = f; *px = wx; *py = wy;
    *dx = len * ox; *dy = len * oy;
    for (int i = 0; i < nc; ++i) {
        double vx = ox, vy = oy;
        rot2(cos(phi[i]), sin(phi[i]), &vx, &vy);
        cx[i] = mag[i] * vx; cy[i] = mag[i] * vy;
    }
}

/* the walk of om_shift; with rec != NULL it also writes the world position of every
 * edge or vertex it crosses (at most cap points; *nrec counts all of them) */
static int shift_rec(const om_mesh* m, int32_t* face, double* bary, const double* disp3,
                     int ncarry, double* carry3, double* rec, int cap, int* nrec) {
    if (ncarry > OM_MAXCARRY) return -1;
    int64_t f = *face;
    double px, py, dx, dy, cx[OM_MAXCARRY], cy[OM_MAXCARRY];
    bary_to_face(m, f, bary, &px, &py);
    world_to_face_vec(m, f, disp3, &dx, &dy);
    for (int i = 0; i < ncarry; ++i) world_to_face_vec(m, f, carry3 + 3 * i, &cx[i], &cy[i]);
    int crossings = 0, entry = -1;
    const double tolb = 1e-12;
    int it;
    for (it = 0; it < 1000000; ++it) {
        double l[3], dl[3];
        bary_of(m, f, px, py, l);
        const double L01 = m->lay[3 * f], x2 = m->lay[3 * f + 1], y2 = m->lay[3 * f + 2];
        dl[2] = dy / y2; dl[1] = (dx - dl[2] * x2) / L01; dl[0] = -dl[1] - dl[2];
        double tmin = OM_INF; int imin = -1;
        for (int i = 0; i < 3; ++i) {
            if (!(dl[i] < 0.0)) continue;
            if ((i + 1) % 3 == entry) continue;        /* never leave through the entry edge */
            double t = -l[i] / dl[i];
            if (t < 0.0) t = 0.0;
            if (t < tmin) { tmin = t; imin = i; }
        }
        if (!(tmin < 1.0)) { px += dx; py += dy; break; }
        const int k = (imin + 1) % 3;                 /* exit edge P_k -> P_{k+1} */
        const double hx = px + tmin * dx, hy = py + tmin * dy;
        double rx = (1.0 - tmin) * dx, ry = (1.0 - tmin) * dy;
        double lh[3];
        bary_of(m, f, hx, hy, lh);
        int vcorner = -1;
        if (lh[(k + 1) % 3] < tolb) vcorner = k;
        else if (lh[k] < tolb) vcorner = (k + 1) % 3;
        ++crossings;
        if (rec) {
            if (*nrec < cap) {
                double w[3];
                face_to_world_vec(m, f, hx, hy, w);
                for (int c = 0; c < 3; ++c) rec[3 * *nrec + c] = m->frame[9 * f + c] + w[c];
            }
            ++*nrec;
        }
        if (vcorner >= 0) {
            vertex_turn(m, &f, vcorner, &px, &py, &rx, &ry, ncarry, cx, cy);
            dx = rx; dy = ry; entry = -1;
            continue;
        }
        const int32_t h = (int32_t)(3 * f + k), tw = m->twin[h];
        double ax, ay, bx, by;
        face_pt(m, f, k, &ax, &ay); face_pt(m, f, k + 1, &bx, &by);
        const double L = hypot(bx - ax, by - ay);
        const double ux = (bx - ax) / L, uy = (by - ay) / L;
        if (tw < 0) {
            /* open boundary: specular reflection of the rest of the step and the carried vectors */
            double pr = dot2(rx, ry, ux, uy);
            rx = 2.0 * pr * ux - rx; ry = 2.0 * pr * uy - ry;
            for (int i = 0; i < ncarry; ++i) {
                double pc = dot2(cx[i], cy[i], ux, uy);
                cx[i] = 2.0 * pc * ux - cx[i]; cy[i] = 2.0 * pc * uy - cy[i];
            }
            px = hx; py = hy; dx = rx; dy = ry; entry = k;
            continue;
        }
        /* unfold into the neighbour: P_k -> Q_{k2+1}, P_{k+1} -> Q_{k2} */
        const int64_t g = tw / 3; const int k2 = tw % 3;
        double qax, qay, qbx, qby;
        face_pt(m, g, k2 + 1, &qax, &qay); face_pt(m, g, k2, &qbx, &qby);
        const double Lg = hypot(qbx - qax, qby - qay);
        const double vx = (qbx - qax) / Lg, vy = (qby - qay) / Lg;
        const double co = dot2(ux, uy, vx, vy), si = cross2(ux, uy, vx, vy);
        double ox = hx - ax, oy = hy - ay;
        rot2(co, si, &ox, &oy);
        px = qax + ox; py = qay + oy;
        rot2(co, si, &rx, &ry);
        for (int i = 0; i < ncarry; ++i) rot2(co, si, &cx[i], &cy[i]);
        dx = rx; dy = ry; f = g; entry = k2;
    }
    if (it >= 1000000) return -2;
    double l[3];
    bary_of(m, f, px, py, l);
    for (int i = 0; i < 3; ++i) if (l[i] < 0.0) l[i] = 0.0;
    const double sum = l[0] + l[1] + l[2];
    for (int i = 0; i < 3; ++i) bary[i] = l[i] / sum;
    *face = (int32_t)f;
    for (int i = 0; i < ncarry; ++i) face_to_world_vec(m, f, cx[i], cy[i], carry3 + 3 * i);
    return crossings;
}

int om_shift(const om_mesh* m, int32_t* face, double* bary, const double* disp3,
             int ncarry, double* carry3) {
    return shift_rec(m, face, bary, disp3, ncarry, carry3, NULL, 0, NULL);
}

/* The straightest geodesic from (face, bary) along the world tangent disp3 (its length is
 * the path length), as a polyline: the start point, every edge or vertex crossing, the end
 * point (world positions, at most cap points; *npts = all points).  face/bary become the
 * end point.  A pair's shortest path is this walk along its initial tangent for its length
 * whenever the path bends at no vertex (Sec. 2.2: shortest paths are straight in the
 * unfolding of the faces they cross). */
int om_trace(const om_mesh* m, int32_t* face, double* bary, const double* disp3, int cap, double* pts,
             int* npts) {
    if (cap > 0) om_world_position(m, *face, bary, pts);
    int n = 1, nrec = 0;
    const int rc = shift_rec(m, face, bary, disp3, 0, NULL, cap > 1 ? pts + 3 : pts, cap > 1 ? cap - 1 : 0, &nrec);
    if (rc < 0) return rc;
    n += nrec;
    if (n < cap) om_world_position(m, *face, bary, pts + 3 * n);
    ++n;
    *npts = n;
    return 0;
}

/* ------------------------------------------------------------------ shortest-path polylines (Sec. 2.2) */
/* A shortest path on the polyhedral surface is a chain of straight legs that meet at
 * pseudo-source vertices (boundary, flat or saddle).  The window propagation above records
 * for every vertex the previous node of its path and, at the query, the last node of the
 * target's path; the path is rebuilt from the target backwards, leg by leg, each leg a
 * straight walk from its start node along the recorded direction for the recorded length. */

static double corner_angle(const om_mesh* m, int64_t f, int k) {
    const int64_t h = 3 * f + k;
    return atan2(m->hcy[h], m->hcx[h]);
}

/* The face of the ring of the vertex at corner k of face f whose wedge holds the direction
 * at angle *phi, counted counter-clockwise from the edge P_k -> P_{k+1} (negative: clockwise
 * of it; beyond the corner angle: past the edge P_k -> P_{k+2}).  Turns face by face around
 * the vertex; on return f, k and *phi refer to that face, with *phi clamped into its
 * wedge.  Returns -1 when the direction leaves the ring through a boundary edge. */
static int ring_locate(const om_mesh* m, int64_t* f, int* k, double* phi) {
    const double tol = 1e-12;
    for (int guard = 0; guard < 256; ++guard) {
        const double a = corner_angle(m, *f, *k);
        if (*phi < -tol) {
            const int32_t tw = m->twin[3 * *f + *k];              /* across P_k -> P_{k+1} */
            if (tw < 0) return -1;
            *f = tw / 3; *k = (tw % 3 + 1) % 3;
            *phi += corner_angle(m, *f, *k);
        } else if (*phi > a + tol) {
            const int32_t tw = m->twin[3 * *f + (*k + 2) % 3];    /* across P_{k+2} -> P_k */
            if (tw < 0) return -1;
            *phi -= a;
            *f = tw / 3; *k = tw % 3;
        } else {
            if (*phi < 0.0) *phi = 0.0;
            if (*phi > a) *phi = a;
            return 0;
        }
    }
    return -1;
}

/* unit direction at angle phi from the edge P_k -> P_{k+1} of face f */
static void corner_dir(const om_mesh* m, int64_t f, int k, double phi, double* dx, double* dy) {
    double ax, ay, bx, by;
    face_pt(m, f, k, &ax, &ay);
    face_pt(m, f, k + 1, &bx, &by);
    const double L = hypot(bx - ax, by - ay);
    double ex = (bx - ax) / L, ey = (by - ay) / L;
    rot2(cos(phi), sin(phi), &ex, &ey);
    *dx = ex; *dy = ey;
}

/* A leg meets a vertex on its way: it goes on straight, i.e. at angle pi from the reversed
 * incoming direction, counted counter-clockwise around the ring if the ring holds that
 * angle on that side, else clockwise (a boundary vertex holds it on one side only). */
static int vertex_pass(const om_mesh* m, int64_t* f, int* k, double* dx, double* dy) {
    double ax, ay, bx, by;
    face_pt(m, *f, *k, &ax, &ay);
    face_pt(m, *f, *k + 1, &bx, &by);
    const double L = hypot(bx - ax, by - ay);
    const double ex = (bx - ax) / L, ey = (by - ay) / L;
    double beta = atan2(cross2(ex, ey, -*dx, -*dy), dot2(ex, ey, -*dx, -*dy));
    const double a = corner_angle(m, *f, *k);
    if (beta < 0.0) beta = 0.0;
    if (beta > a) beta = a;
    int64_t g = *f; int kg = *k;
    double phi = beta + OM_PI;
    if (ring_locate(m, &g, &kg, &phi) < 0) {
        g = *f; kg = *k; phi = beta - OM_PI;
        if (ring_locate(m, &g, &kg, &phi) < 0) return -1;
    }
    *f = g; *k = kg;
    corner_dir(m, g, kg, phi, dx, dy);
    return 0;
}

/* Straight walk of one leg: from corner kc of face f (kc >= 0; the unit direction (dx, dy)
 * of f's layout may point into any face of the vertex's ring) or from the point (px, py) of
 * f (kc < 0), for length len.  Every edge or vertex crossed before the end is written to
 * rec (world positions, at most cap, *nrec counts all); the end point is returned as face
 * *fend and layout point (*ex, *ey).  A crossing within 1e-12 of the leg's end is the end. */
static int leg_walk(const om_mesh* m, int64_t f, int kc, double px, double py, double dx, double dy, double len,
                    double* rec, int cap, int* nrec, int64_t* fend, double* ex, double* ey) {
    int corner = kc;
    if (corner < 0) {   /* a start point on a corner of its face starts from that vertex */
        double l[3];
        bary_of(m, f, px, py, l);
        for (int c = 0; c < 3; ++c)
            if (l[c] > 1.0 - 1e-12) corner = c;
    }
    if (corner >= 0) {
        double ax, ay, bx, by;
        face_pt(m, f, corner, &ax, &ay);
        face_pt(m, f, corner + 1, &bx, &by);
        const double L = hypot(bx - ax, by - ay);
        const double ux = (bx - ax) / L, uy = (by - ay) / L;
        double phi = atan2(cross2(ux, uy, dx, dy), dot2(ux, uy, dx, dy));
        if (ring_locate(m, &f, &corner, &phi) < 0) return -3;
        corner_dir(m, f, corner, phi, &dx, &dy);
        face_pt(m, f, corner, &px, &py);
    }
    double rem = len;
    int entry = -1;
    const double tolb = 1e-12;
    int it;
    for (it = 0; it < 1000000; ++it) {
        double l[3], dl[3];
        bary_of(m, f, px, py, l);
        const double Dx = dx * rem, Dy = dy * rem;
        const double L01 = m->lay[3 * f], x2 = m->lay[3 * f + 1], y2 = m->lay[3 * f + 2];
        dl[2] = Dy / y2; dl[1] = (Dx - dl[2] * x2) / L01; dl[0] = -dl[1] - dl[2];
        double tmin = OM_INF; int imin = -1;
        for (int i = 0; i < 3; ++i) {
            if (corner >= 0 && i != corner) continue;   /* from a corner: only the far edge */
            if (!(dl[i] < 0.0)) continue;
            if ((i + 1) % 3 == entry) continue;
            double t = -l[i] / dl[i];
            if (t < 0.0) t = 0.0;
            if (t < tmin) { tmin = t; imin = i; }
        }
        if (!(tmin < 1.0 - 1e-12)) { px += Dx; py += Dy; break; }
        const int k = (imin + 1) % 3;
        const double hx = px + tmin * Dx, hy = py + tmin * Dy;
        rem *= (1.0 - tmin);
        double lh[3];
        bary_of(m, f, hx, hy, lh);
        int vcorner = -1;
        if (lh[(k + 1) % 3] < tolb) vcorner = k;
        else if (lh[k] < tolb) vcorner = (k + 1) % 3;
        if (rec && *nrec < cap) {
            double w[3];
            if (vcorner >= 0) { double vx, vy; face_pt(m, f, vcorner, &vx, &vy); face_to_world_vec(m, f, vx, vy, w); }
            else face_to_world_vec(m, f, hx, hy, w);
            for (int c = 0; c < 3; ++c) rec[3 * *nrec + c] = m->frame[9 * f + c] + w[c];
        }
        if (rec) ++*nrec;
        if (vcorner >= 0) {
            int kk = vcorner;
            if (vertex_pass(m, &f, &kk, &dx, &dy) < 0) return -4;
            corner = kk;
            face_pt(m, f, corner, &px, &py);
            entry = -1;
            continue;
        }
        const int32_t h = (int32_t)(3 * f + k), tw = m->twin[h];
        if (tw < 0) return -5;    /* a shortest path never crosses the boundary */
        double ax, ay, bx, by;
        face_pt(m, f, k, &ax, &ay); face_pt(m, f, k + 1, &bx, &by);
        const double L = hypot(bx - ax, by - ay);
        const double ux = (bx - ax) / L, uy = (by - ay) / L;
        const int64_t g = tw / 3; const int k2 = tw % 3;
        double qax, qay, qbx, qby;
        face_pt(m, g, k2 + 1, &qax, &qay); face_pt(m, g, k2, &qbx, &qby);
        const double Lg = hypot(qbx - qax, qby - qay);
        const double vx = (qbx - qax) / Lg, vy = (qby - qay) / Lg;
        const double co = dot2(ux, uy, vx, vy), si = cross2(ux, uy, vx, vy);
        double ox = hx - ax, oy = hy - ay;
        rot2(co, si, &ox, &oy);
        px = qax + ox; py = qay + oy;
        rot2(co, si, &dx, &dy);
        f = g; entry = k2; corner = -1;
    }
    if (it >= 1000000) return -2;
    *fend = f; *ex = px; *ey = py;
    return 0;
}

static void layout_world(const om_mesh* m, int64_t f, double x, double y, double* out3) {
    double w[3];
    face_to_world_vec(m, f, x, y, w);
    for (int c = 0; c < 3; ++c) out3[c] = m->frame[9 * f + c] + w[c];
}

static void wrap_world(const om_mesh* m, double* p) {
    if (m->periodic)
        for (int a = 0; a < 2; ++a) p[a] -= m->per[a] * floor(p[a] / m->per[a]);
}

#define OM_MAXLEGS 64

int om_geodesic_paths(const om_mesh* m, int64_t n, const int32_t* face, const double* bary, double r_c,
                      int64_t np, const int32_t* src, const int32_t* dst, int cap, double* pts, int32_t* npts,
                      int32_t* nlegs, double* dist, double* gap) {
    ows* s = ws_create(m);
    s->rc = r_c;
    int32_t cur = -1;
    double* buf = (double*)malloc(sizeof(double) * 3 * (size_t)(cap > 0 ? cap : 1));
    int rc_all = 0;
    for (int64_t p = 0; p < np; ++p) {
        const int32_t i = src[p], j = dst[p];
        npts[p] = 0; nlegs[p] = 0; dist[p] = OM_INF; gap[p] = 0.0;
        if (i < 0 || i >= n || j < 0 || j >= n || i == j) { rc_all = -1; continue; }
        if (i != cur) { run_source(s, face[i], bary + 3 * (int64_t)i); cur = i; }
        double qx, qy, tx, ty;
        bary_to_face(m, face[i], bary + 3 * (int64_t)i, &qx, &qy);
        olink lk;
        const double d = query_point_c(s, face[i], qx, qy, face[j], bary + 3 * (int64_t)j, &tx, &ty, NULL, &lk);
        if (!(d < r_c)) continue;
        dist[p] = d;
        /* walk back from the target: its leg, then each node's leg until the source */
        int nb = 0, legs = 0;
        double e[3];
        om_world_position(m, face[j], bary + 3 * (int64_t)j, e);
        if (nb < cap) memcpy(buf + 3 * nb, e, sizeof(e));
        ++nb;
        double sx, sy;
        bary_to_face(m, face[j], bary + 3 * (int64_t)j, &sx, &sy);
        int64_t f = face[j]; int kc = -1;
        double g = 0.0;
        for (;;) {
            if (legs >= OM_MAXLEGS) { rc_all = -6; break; }
            int nrec = 0;
            int64_t fe; double ex, ey;
            const int w = leg_walk(m, f, kc, sx, sy, lk.dx, lk.dy, lk.len, buf + 3 * (nb < cap ? nb : 0),
                                   nb < cap ? cap - nb : 0, &nrec, &fe, &ex, &ey);
            if (w < 0) { rc_all = w; break; }
            for (int r = 0; r < nrec && nb + r < cap; ++r) wrap_world(m, buf + 3 * (nb + r));
            nb += nrec;
            ++legs;
            /* where the leg should have ended: the next node */
            double node[3], end[3];
            layout_world(m, fe, ex, ey, end);
            if (lk.par < 0) om_world_position(m, face[i], bary + 3 * (int64_t)i, node);
            else {
                const int32_t v = lk.par;
                double vx, vy;
                face_pt(m, s->pf[v], s->pc[v], &vx, &vy);
                layout_world(m, s->pf[v], vx, vy, node);
            }
            double dd[3] = {end[0] - node[0], end[1] - node[1], end[2] - node[2]};
            min_image(m, dd);
            const double gl = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            if (gl > g) g = gl;
            wrap_world(m, node);
            if (nb < cap) memcpy(buf + 3 * nb, node, sizeof(node));
            ++nb;
            if (lk.par < 0) break;
            const int32_t v = lk.par;
            f = s->pf[v]; kc = s->pc[v];
            lk.par = s->par[v]; lk.dx = s->pdir[2 * v]; lk.dy = s->pdir[2 * v + 1]; lk.len = s->plen[v];
        }
        /* source first */
        const int kept = nb < cap ? nb : cap;
        for (int r = 0; r < kept; ++r)
            for (int c = 0; c < 3; ++c) pts[3 * ((int64_t)p * cap + r) + c] = buf[3 * (kept - 1 - r) + c];
        npts[p] = nb; nlegs[p] = legs; gap[p] = g;
    }
    free(buf);
    ws_destroy(s);
    return rc_all;
}

/* ------------------------------------------------------------------ Philox4x32-10 (Salmon et al.) */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32); *lo = (uint32_t)p;
}

void om_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* two standard normals for (seed, particle, step): Box-Muller on two 53-bit uniforms */
void om_normal_pair(uint64_t seed, uint64_t particle, uint64_t step, double* z0, double* z1) {
    uint32_t ctr[4] = {(uint32_t)particle, (uint32_t)(particle >> 32), (uint32_t)step, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    om_philox4x32_10(ctr, key, o);
    const double u1 = ((double)(o[0] >> 5) * 67108864.0 + (double)(o[1] >> 6) + 0.5) / 9007199254740992.0;
    const double u2 = ((double)(o[2] >> 5) * 67108864.0 + (double)(o[3] >> 6) + 0.5) / 9007199254740992.0;
    const double r = sqrt(-2.0 * log(u1));
    *z0 = r * cos(2.0 * OM_PI * u2);
    *z1 = r * sin(2.0 * OM_PI * u2);
}

/* ------------------------------------------------------------------ dynamics (Sec. 2.1) */
static void clamp_disp(double* d, double maxd) {
    const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (n > maxd) for (int a = 0; a < 3; ++a) d[a] *= maxd / n;
}

int om_integrate(const om_mesh* m, int64_t n, int32_t* face, double* bary, double* vel,
                 double* orient, double* force, const om_potential* pot,
                 const om_integrator* it, double r_c, int64_t nsteps, uint64_t seed,
                 int64_t step0, const double* noise, double* epot, int nthreads) {
    int rc = 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        const uint64_t step = (uint64_t)(step0 + s);
        if (it->kind == 0) {
            /* velocity Verlet: half kick, geodesic drift carrying v, new forces, half kick */
            const double h = 0.5 * it->dt / it->mass;
            for (int64_t i = 0; i < n; ++i) {
                double d[3];
                for (int a = 0; a < 3; ++a) { vel[3 * i + a] += h * force[3 * i + a]; d[a] = it->dt * vel[3 * i + a]; }
                clamp_disp(d, it->max_disp);
                if (om_shift(m, face + i, bary + 3 * i, d, 1, vel + 3 * i) < 0) return -6;
            }
            rc = om_forces(m, n, face, bary, r_c, pot, force, epot, nthreads);
            if (rc) return rc;
            for (int64_t i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) vel[3 * i + a] += h * force[3 * i + a];
        } else if (it->kind == 3) {
            /* steepest descent (the relaxation of Fig. 3): dr = (dt / lambda) f, no noise */
            rc = om_forces(m, n, face, bary, r_c, pot, force, epot, nthreads);
            if (rc) return rc;
            for (int64_t i = 0; i < n; ++i) {
                double d[3];
                for (int a = 0; a < 3; ++a) d[a] = it->dt / it->lam * force[3 * i + a];
                clamp_disp(d, it->max_disp);
                if (om_shift(m, face + i, bary + 3 * i, d, 0, NULL) < 0) return -6;
            }
        } else {
            rc = om_forces(m, n, face, bary, r_c, pot, force, epot, nthreads);
            if (rc) return rc;
            for (int64_t i = 0; i < n; ++i) {
                double z0, z1;
                if (noise) { z0 = noise[2 * (s * n + i)]; z1 = noise[2 * (s * n + i) + 1]; }
                else om_normal_pair(seed, (uint64_t)i, step, &z0, &z1);
                const double* fr = m->frame + 9 * (int64_t)face[i];
                double d[3];
                if (it->kind == 1) {
                    /* Brownian: lambda dr = dt f + sqrt(2 kT lambda dt) eta, eta in the face plane */
                    const double amp = sqrt(2.0 * it->kT * it->dt / it->lam);
                    for (int a = 0; a < 3; ++a)
                        d[a] = it->dt / it->lam * force[3 * i + a] + amp * (z0 * fr[3 + a] + z1 * fr[6 + a]);
                    clamp_disp(d, it->max_disp);
                    if (om_shift(m, face + i, bary + 3 * i, d, 0, NULL) < 0) return -6;
                } else {
                    /* active Brownian: dr = dt (v0 n + f / lambda); n transported, then rotated */
                    for (int a = 0; a < 3; ++a)
                        d[a] = it->dt * (it->v0 * orient[3 * i + a] + force[3 * i + a] / it->lam);
                    clamp_disp(d, it->max_disp);
                    if (om_shift(m, face + i, bary + 3 * i, d, 1, orient + 3 * i) < 0) return -6;
                    const double* g = m->frame + 9 * (int64_t)face[i];
                    double ox, oy;
                    world_to_face_vec(m, face[i], orient + 3 * i, &ox, &oy);
                    const double on = hypot(ox, oy);
                    ox /= on; oy /= on;
                    rot2(cos(sqrt(2.0 * it->Dr * it->dt) * z0), sin(sqrt(2.0 * it->Dr * it->dt) * z0), &ox, &oy);
                    for (int a = 0; a < 3; ++a) orient[3 * i + a] = ox * g[3 + a] + oy * g[6 + a];
                }
            }
        }
    }
    return rc;
}

/* ------------------------------------------------------------------ FIRE minimiser
 * Fast inertial relaxation (Bitzek et al., PRL 97, 170201, 2006) on the surface: each step
 * (1) P = sum_i f_i . v_i; (2) v_i <- (1 - alpha) v_i + alpha |v| f_i / |f| with the norms of
 * the whole system's vectors; (3) if P > 0 count it, and after more than N_min such steps
 * in a row grow dt (x f_inc, at most dt_max) and shrink alpha (x f_alpha); (4) if P <= 0
 * halve dt, set v = 0, alpha = alpha_start and restart the count; then one velocity-Verlet
 * step with the current dt (drift = face walk carrying v). Forces must hold the forces at
 * the current positions on entry and hold them at the final positions on exit.
 * state[3] = {dt, alpha, steps with P > 0} in/out. */
int om_fire(const om_mesh* m, int64_t n, int32_t* face, double* bary, double* vel, double* force,
            const om_potential* pot, const om_integrator* it, double r_c, int64_t nsteps, double* state,
            double* epot, int nthreads) {
    const double alpha0 = OM_FIRE_ALPHA0, f_inc = OM_FIRE_FINC, f_dec = OM_FIRE_FDEC, f_alpha = OM_FIRE_FALPHA;
    const double dt_max = OM_FIRE_DTMAX * it->dt;
    for (int64_t s = 0; s < nsteps; ++s) {
        double P = 0.0, vv = 0.0, ff = 0.0;
        for (int64_t i = 0; i < 3 * n; ++i) { P += force[i] * vel[i]; vv += vel[i] * vel[i]; ff += force[i] * force[i]; }
        const double alpha = state[1];
        if (ff > 0.0) {
            const double c = alpha * sqrt(vv) / sqrt(ff);
            for (int64_t i = 0; i < 3 * n; ++i) vel[i] = (1.0 - alpha) * vel[i] + c * force[i];
        }
        if (P > 0.0) {
            state[2] += 1.0;
            if (state[2] > OM_FIRE_NMIN) {
                state[0] = fmin(state[0] * f_inc, dt_max);
                state[1] = alpha * f_alpha;
            }
        } else {
            state[2] = 0.0;
            state[0] *= f_dec;
            state[1] = alpha0;
            for (int64_t i = 0; i < 3 * n; ++i) vel[i] = 0.0;
        }
        const double dt = state[0], h = 0.5 * dt / it->mass;
        for (int64_t i = 0; i < n; ++i) {
            double d[3];
            for (int a = 0; a < 3; ++a) { vel[3 * i + a] += h * force[3 * i + a]; d[a] = dt * vel[3 * i + a]; }
            clamp_disp(d, it->max_disp);
            if (om_shift(m, face + i, bary + 3 * i, d, 1, vel + 3 * i) < 0) return -6;
        }
        const int rc = om_forces(m, n, face, bary, r_c, pot, force, epot, nthreads);
        if (rc) return rc;
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += h * force[i];
    }
    return 0;
}
