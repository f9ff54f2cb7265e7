/*
 * mpm_oracle.c -- plain, single-threaded FP64 reference of one MLS-MPM time
 * step with a Neo-Hookean material and rigid-tool collision handling, written
 * from Sec. III-B (Eqs. 1-10) and Sec. III-C (Eqs. 11-19) of "Efficient
 * Physically-based Simulation of Soft Bodies in Embodied Environment for
 * Surgical Robot" (Yang et al., arXiv 2402.01181).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA library:
 * only the tests, the package smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no source, header, table or helper with the CUDA
 * path, and the CUDA path never links or calls it.
 *
 * Everything is written in the order and notation of the paper: a step is
 * P2G (Eqs. 1-3, with Eq. 5-6 for the stress), the grid operation (Eq. 7,
 * boundary conditions, Eqs. 11-19 for tools), then G2P and advection
 * (Eqs. 8-10, with Eq. 4 for F).  No blocking, sorting or fusion.
 *
 * Readings where the paper is silent or garbled (each listed in the design
 * notes of the repository):
 *   - Eq. 5 prints mu(F - F^T); the Neo-Hookean first Piola stress of the
 *     cited MLS-MPM references is P = mu(F - F^-T) + lambda ln(J) F^-T, which
 *     is what is evaluated here ("log" is the natural logarithm).
 *   - Eq. 3 multiplies P(F') by F_p^T; the F stored on a particle is the one
 *     already updated by Eq. 4 at the end of the previous G2P, so the stress
 *     term uses P(F) F^T of that stored F.
 *   - Quadratic B-spline weights (the paper defers w_ip to its references).
 *   - Grid velocity is formed only where m_i > 0; gravity is added after
 *     Eq. 7; sticky walls zero every component at nodes within `bound` nodes
 *     of the domain faces, applied after tool handling.
 *   - Tools use analytic distance functions (capsule, box) with their
 *     analytic, normalised gradients, or a sampled distance field (Eqs. 12-14)
 *     read at the sample floor((x_ref - o) / h) with the central-difference
 *     normal of Eq. 14 (one-sided at the faces of the volume), normalised;
 *     points outside the sampled volume are not in contact; the
 *     friction update of Eq. 18 is clamped at zero tangential speed; nodes
 *     with v_n >= 0 are left unchanged; several tools are merged by minimum
 *     distance with the lowest tool index winning ties (the z-buffer of
 *     Sec. III-C).
 *   - J <= 0 is clamped to 1e-6 inside ln and counted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n_grid;       /* nodes per axis; domain [0,1)^3, dx = 1/n_grid */
    int32_t bound;        /* sticky wall band, in nodes */
    double dt;            /* Delta t */
    double gravity[3];
    double E, nu, rho;    /* Young's modulus, Poisson ratio, density */
    double V0;            /* V_p^0, equal for every particle; m_p = rho V_p^0 */
    double theta;         /* collision threshold: contact if distance < theta */
    double friction;      /* Coulomb coefficient mu of Eq. 18 */
} orc_params;

/* One rigid tool at one sub-step: world position of a reference-frame point
 * is x = R x_ref + T (Eq. 11 inverts this). */
typedef struct {
    int32_t kind;         /* 0 capsule: dims = (radius, half-length along local y); 1 box: half extents;
                             2 sampled distance field: dims = reference-frame position of sample (0,0,0) */
    int32_t res;          /* kind 2: samples per axis */
    double dims[3];
    double R[9];          /* row-major rotation */
    double T[3];
    double u[3];          /* linear velocity of the reference point T */
    double w[3];          /* angular velocity */
    double h;             /* kind 2: sample spacing (the dx of Eq. 13) */
    const float *sdf;     /* kind 2: res^3 samples, sample (i,j,k) at sdf[(k res + j) res + i]
                             holds the distance at dims + h (i, j, k) */
} orc_tool;

typedef struct {
    int64_t j_clamped;    /* particles whose J <= 0 was clamped */
    int64_t out_of_domain;/* particles whose stencil left the grid (clamped) */
} orc_counters;

/* ---------------------------------------------------------------- algebra */

static void mat_mul(const double *A, const double *B, double *C) /* C = A B */
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static double mat_det(const double *A)
{
    return A[0] * (A[4] * A[8] - A[5] * A[7])
         - A[1] * (A[3] * A[8] - A[5] * A[6])
         + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* inverse transpose via the cofactor matrix: A^-T = cof(A) / det(A) */
static void mat_inv_transpose(const double *A, double det, double *out)
{
    out[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    out[1] = -(A[3] * A[8] - A[5] * A[6]) / det;
    out[2] = (A[3] * A[7] - A[4] * A[6]) / det;
    out[3] = -(A[1] * A[8] - A[2] * A[7]) / det;
    out[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    out[5] = -(A[0] * A[7] - A[1] * A[6]) / det;
    out[6] = (A[1] * A[5] - A[2] * A[4]) / det;
    out[7] = -(A[0] * A[5] - A[2] * A[3]) / det;
    out[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

/* ------------------------------------------------------ material (Eq. 5-6) */

/* Eq. 6: Lame parameters from Young's modulus and Poisson's ratio. */
void orc_lame(double E, double nu, double *mu, double *lam)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* Eq. 5 (reading: F^-T in the first term): first Piola-Kirchhoff stress.
 * Returns 1 if J <= 0 had to be clamped inside ln. */
int orc_piola(double mu, double lam, const double *F, double *P)
{
    double J = mat_det(F);
    int clamped = 0;
    double lnJ;
    if (J <= 0.0) { clamped = 1; lnJ = log(1e-6); } else lnJ = log(J);
    double FiT[9];
    if (J == 0.0) { /* no inverse: fall back to the identity so P stays finite */
        for (int i = 0; i < 9; ++i) FiT[i] = (i % 4 == 0) ? 1.0 : 0.0;
    } else {
        mat_inv_transpose(F, J, FiT);
    }
    for (int i = 0; i < 9; ++i) P[i] = mu * (F[i] - FiT[i]) + lam * lnJ * FiT[i];
    return clamped;
}

/* P(F) F^T, the product that enters Eq. 3. */
int orc_piola_FT(double mu, double lam, const double *F, double *out)
{
    double P[9], FT[9];
    int c = orc_piola(mu, lam, F, P);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) FT[3 * i + j] = F[3 * j + i];
    mat_mul(P, FT, out);
    return c;
}

/* ---------------------------------------------- quadratic B-spline weights */

/* For one axis, with fx = x/dx - base in [0.5, 1.5), the weights of the nodes
 * base, base+1, base+2 (the kernel the paper's references use for w_ip). */
void orc_weights(double fx, double *w)
{
    w[0] = 0.5 * (1.5 - fx) * (1.5 - fx);
    w[1] = 0.75 - (fx - 1.0) * (fx - 1.0);
    w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);
}

static int stencil_base(const orc_params *p, const double *xp, int *base, double *fx)
{
    int bad = 0;
    for (int d = 0; d < 3; ++d) {
        double s = xp[d] * (double)p->n_grid;
        int b = (int)floor(s - 0.5);
        if (b < 0) { b = 0; bad = 1; }
        if (b > p->n_grid - 3) { b = p->n_grid - 3; bad = 1; }
        base[d] = b;
        fx[d] = s - (double)b;
    }
    return bad;
}

static inline int64_t node_index(int n, int i, int j, int k)
{
    return ((int64_t)i * n + j) * n + k;   /* grid[i][j][k], k fastest */
}

/* ------------------------------------------------------------ P2G (Eq. 1-3) */

/* Scatter particle mass and momentum to the grid.  grid_m: n^3, grid_mv:
 * n^3 x 3, both overwritten.  x, v: N x 3; C, F: N x 9 row-major. */
void orc_p2g(const orc_params *p, int64_t N, const double *x, const double *v,
             const double *C, const double *F, double *grid_m, double *grid_mv,
             orc_counters *cnt)
{
    const int n = p->n_grid;
    const double dx = 1.0 / n;
    const double mp = p->rho * p->V0;
    double mu, lam;
    orc_lame(p->E, p->nu, &mu, &lam);
    const int64_t nn = (int64_t)n * n * n;
    memset(grid_m, 0, sizeof(double) * nn);
    memset(grid_mv, 0, sizeof(double) * nn * 3);

    for (int64_t q = 0; q < N; ++q) {
        const double *xp = x + 3 * q, *vp = v + 3 * q, *Cp = C + 9 * q, *Fp = F + 9 * q;
        int base[3];
        double fx[3], w[3][3];
        if (stencil_base(p, xp, base, fx) && cnt) cnt->out_of_domain++;
        for (int d = 0; d < 3; ++d) orc_weights(fx[d], w[d]);
        double PFt[9];
        int c = orc_piola_FT(mu, lam, Fp, PFt);
        if (c && cnt) cnt->j_clamped++;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const double wip = w[0][i] * w[1][j] * w[2][k];
                    const double xi_xp[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (k - fx[2]) * dx};
                    double mom[3];
                    for (int a = 0; a < 3; ++a) {
                        double Cd = 0.0, Sd = 0.0;
                        for (int b = 0; b < 3; ++b) {
                            Cd += Cp[3 * a + b] * xi_xp[b];
                            Sd += PFt[3 * a + b] * xi_xp[b];
                        }
                        /* Eq. 3: f_ip = -(4/dx^2) V_p^0 P(F) F^T (x_i - x_p) */
                        const double f = -(4.0 / (dx * dx)) * p->V0 * Sd;
                        /* Eq. 1: m_p v_p + m_p C_p (x_i - x_p) + f_ip dt */
                        mom[a] = mp * vp[a] + mp * Cd + f * p->dt;
                    }
                    const int64_t I = node_index(n, base[0] + i, base[1] + j, base[2] + k);
                    for (int a = 0; a < 3; ++a) grid_mv[3 * I + a] += wip * mom[a];
                    grid_m[I] += wip * mp;      /* Eq. 2 */
                }
    }
}

/* -------------------------------------------------- tool geometry (Eq. 11) */

/* Rodrigues: rotation matrix of the rotation vector r. */
void orc_rotvec_to_matrix(const double *r, double *R)
{
    const double th = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const double K[9] = {0, -r[2], r[1], r[2], 0, -r[0], -r[1], r[0], 0};
    double K2[9];
    mat_mul(K, K, K2);
    double a, b;
    if (th < 1e-8) { a = 1.0 - th * th / 6.0; b = 0.5 - th * th / 24.0; }
    else { a = sin(th) / th; b = (1.0 - cos(th)) / (th * th); }
    for (int i = 0; i < 9; ++i) R[i] = ((i % 4 == 0) ? 1.0 : 0.0) + a * K[i] + b * K2[i];
}

/* Inverse of Rodrigues for angles in [0, pi]. */
void orc_matrix_to_rotvec(const double *R, double *r)
{
    const double tr = R[0] + R[4] + R[8];
    double c = 0.5 * (tr - 1.0);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    const double th = acos(c);
    const double s[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};  /* 2 sin(th) axis */
    if (th < 1e-8) {
        for (int d = 0; d < 3; ++d) r[d] = 0.5 * s[d];
        return;
    }
    if (th < 3.14159265358979323846 - 1e-6) {
        const double f = th / (2.0 * sin(th));
        for (int d = 0; d < 3; ++d) r[d] = f * s[d];
        return;
    }
    /* near pi: axis from the symmetric part R = 2 a a^T - I */
    double a[3];
    for (int d = 0; d < 3; ++d) {
        double v = 0.5 * (R[4 * d] + 1.0);
        a[d] = v > 0.0 ? sqrt(v) : 0.0;
    }
    int m = 0;
    if (a[1] > a[m]) m = 1;
    if (a[2] > a[m]) m = 2;
    for (int d = 0; d < 3; ++d)
        if (d != m) {
            double sym = 0.5 * (R[3 * m + d] + R[3 * d + m]);
            a[d] = sym / (2.0 * a[m]);
        }
    double nrm = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    for (int d = 0; d < 3; ++d) r[d] = th * a[d] / nrm;
}

/* Tool frames for the sub-steps of one call that moves a tool uniformly from
 * pose0 to pose1 (6-vectors: T, rotation vector) over nsub sub-steps of dt.
 * Sub-step k uses the pose at fraction s = (k+1)/nsub:
 *   T_k = T0 + s (T1 - T0),  R_k = exp(s phi) R0 with phi = log(R1 R0^T),
 * and the rigid velocity field u + w x (x - T_k) with u = (T1 - T0)/(nsub dt),
 * w = phi/(nsub dt).  With nsub = 1 this is the finite difference of
 * consecutive poses. */
void orc_tool_frames(int32_t kind, const double *dims, const double *pose0,
                     const double *pose1, int32_t nsub, double dt, orc_tool *out)
{
    double R0[9], R1[9], R0T[9], Rrel[9], phi[3];
    orc_rotvec_to_matrix(pose0 + 3, R0);
    orc_rotvec_to_matrix(pose1 + 3, R1);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R0T[3 * i + j] = R0[3 * j + i];
    mat_mul(R1, R0T, Rrel);
    orc_matrix_to_rotvec(Rrel, phi);
    const double span = nsub * dt;
    for (int k = 0; k < nsub; ++k) {
        const double s = (double)(k + 1) / (double)nsub;
        orc_tool *t = out + k;
        t->kind = kind;
        t->res = 0;
        t->h = 0.0;
        t->sdf = NULL;
        for (int d = 0; d < 3; ++d) t->dims[d] = dims[d];
        double rs[3] = {s * phi[0], s * phi[1], s * phi[2]}, Rs[9];
        orc_rotvec_to_matrix(rs, Rs);
        mat_mul(Rs, R0, t->R);
        for (int d = 0; d < 3; ++d) {
            t->T[d] = pose0[d] + s * (pose1[d] - pose0[d]);
            t->u[d] = (pose1[d] - pose0[d]) / span;
            t->w[d] = phi[d] / span;
        }
    }
}

/* Signed distance of a reference-frame point to the tool surface and the
 * outward unit normal there (analytic stand-in for Eqs. 12-14). */
double orc_sdf(int32_t kind, const double *dims, const double *p, double *nrm)
{
    if (kind == 0) {                  /* capsule around the local y segment */
        double c = p[1];
        if (c > dims[1]) c = dims[1];
        if (c < -dims[1]) c = -dims[1];
        const double q[3] = {p[0], p[1] - c, p[2]};
        const double L = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (L > 0.0) { nrm[0] = q[0] / L; nrm[1] = q[1] / L; nrm[2] = q[2] / L; }
        else { nrm[0] = 0.0; nrm[1] = 1.0; nrm[2] = 0.0; }
        return L - dims[0];
    }
    /* box with half extents dims */
    double q[3], o[3], on = 0.0;
    for (int d = 0; d < 3; ++d) {
        q[d] = fabs(p[d]) - dims[d];
        o[d] = q[d] > 0.0 ? q[d] : 0.0;
        on += o[d] * o[d];
    }
    on = sqrt(on);
    if (on > 0.0) {
        for (int d = 0; d < 3; ++d) nrm[d] = (p[d] < 0.0 ? -1.0 : 1.0) * o[d] / on;
        return on;
    }
    int a = 0;
    if (q[1] > q[a]) a = 1;
    if (q[2] > q[a]) a = 2;
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    nrm[a] = p[a] < 0.0 ? -1.0 : 1.0;
    return q[a];
}

/* Sampled distance field, Eqs. 12-14.  Eq. 12 indexes the precomputed field
 * by x_ref / dx; with the field's first sample at o the index of a
 * reference-frame point is floor((p - o) / h) on each axis.  The distance is
 * that sample; the normal is Eq. 14's central difference of the neighbouring
 * samples (a one-sided difference where the neighbour would lie outside the
 * field), normalised.  Returns +inf outside the field.  cell_margin (optional):
 * distance of p from the nearest cell face, the floor decision's margin. */
double orc_sdf_sampled(const float *sdf, int32_t res, const double *o, double h,
                       const double *p, double *nrm, double *cell_margin)
{
    int64_t c[3];
    double cm = INFINITY;
    for (int a = 0; a < 3; ++a) {
        const double u = (p[a] - o[a]) / h;
        const double f = floor(u);
        const double gap = (u - f < f + 1.0 - u ? u - f : f + 1.0 - u) * h;
        if (gap < cm) cm = gap;
        if (!(f >= 0.0 && f < (double)res)) {
            if (cell_margin) *cell_margin = cm;
            nrm[0] = 0.0; nrm[1] = 1.0; nrm[2] = 0.0;
            return INFINITY;
        }
        c[a] = (int64_t)f;
    }
    if (cell_margin) *cell_margin = cm;
#define ORC_SDF_AT(i, j, k) ((double)sdf[((int64_t)(k) * res + (j)) * res + (i)])
    double g[3];
    for (int a = 0; a < 3; ++a) {
        int64_t lo[3] = {c[0], c[1], c[2]}, hi[3] = {c[0], c[1], c[2]};
        if (lo[a] > 0) lo[a] -= 1;
        if (hi[a] < res - 1) hi[a] += 1;
        const double span = (double)(hi[a] - lo[a]) * h;
        g[a] = span > 0.0 ? (ORC_SDF_AT(hi[0], hi[1], hi[2]) - ORC_SDF_AT(lo[0], lo[1], lo[2])) / span : 0.0;
    }
    const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gn > 0.0) { nrm[0] = g[0] / gn; nrm[1] = g[1] / gn; nrm[2] = g[2] / gn; }
    else { nrm[0] = 0.0; nrm[1] = 1.0; nrm[2] = 0.0; }
    const double d = ORC_SDF_AT(c[0], c[1], c[2]);
#undef ORC_SDF_AT
    return d;
}

/* ------------------------------------------- grid operation (Eq. 7, 11-19) */

/* What the contact response of one node computed (Eqs. 15-19), kept for the
 * margins and for the adjoint. */
typedef struct {
    double nw[3];         /* world unit normal R nref */
    double r[3];          /* x - T */
    double vco[3];        /* rigid tool velocity at the node */
    double vrel[3];       /* Eq. 15 */
    double vn;            /* Eq. 16 */
    double vt[3];         /* Eq. 17 */
    double vtn;           /* |v_t| */
    double s;             /* |v_t| + mu_f v_n, the unclamped Eq. 18 length */
    double scale;         /* clamped Eq. 18 factor on v_t */
    int projected;        /* v_n < 0: Eqs. 17-19 applied */
} orc_contact;

/* z-buffer of Sec. III-C at the world node position xw: the tool with the
 * smallest distance (lowest index on ties).  Returns that distance (+inf if
 * no tool); *id, nref and xref receive the tool, its reference-frame normal
 * and the node's reference-frame position; *d2 the second-smallest distance;
 * *cells (if given) the smallest sample-cell margin of a sampled field whose
 * sample lies within 2h of theta. */
static double nearest_tool(const orc_tool *tools, int32_t ntools, double theta, const double *xw,
                           int *id, double *nref, double *xref, double *d2, double *cells)
{
    double dmin = INFINITY;
    *id = -1;
    *d2 = INFINITY;
    if (cells) *cells = INFINITY;
    for (int t = 0; t < ntools; ++t) {
        const orc_tool *tl = tools + t;
        double xr[3], nr[3];
        for (int a = 0; a < 3; ++a) {   /* Eq. 11: R^-1 (x - T) */
            double s = 0.0;
            for (int b = 0; b < 3; ++b) s += tl->R[3 * b + a] * (xw[b] - tl->T[b]);
            xr[a] = s;
        }
        double cm = INFINITY;
        const double d = tl->kind == 2 ? orc_sdf_sampled(tl->sdf, tl->res, tl->dims, tl->h, xr, nr, &cm)
                                       : orc_sdf(tl->kind, tl->dims, xr, nr);
        /* a neighbouring sample of a distance field differs by at most
           sqrt(3) h, so the cell decision matters only near contact */
        if (cells && d < theta + 2.0 * tl->h && cm < *cells) *cells = cm;
        if (d < dmin) {
            *d2 = dmin;
            dmin = d; *id = t;
            for (int a = 0; a < 3; ++a) { nref[a] = nr[a]; xref[a] = xr[a]; }
        } else if (d < *d2) {
            *d2 = d;
        }
    }
    return dmin;
}

/* Eqs. 15-19 at a node at xw in contact with tool tl whose reference-frame
 * normal is nref: v is replaced by the response (unchanged if separating). */
static void contact_response(const orc_params *p, const orc_tool *tl, const double *xw, const double *nref,
                             double *v, orc_contact *c)
{
    for (int a = 0; a < 3; ++a) {
        c->nw[a] = 0.0;
        for (int b = 0; b < 3; ++b) c->nw[a] += tl->R[3 * a + b] * nref[b];
        c->r[a] = xw[a] - tl->T[a];
    }
    c->vco[0] = tl->u[0] + tl->w[1] * c->r[2] - tl->w[2] * c->r[1];
    c->vco[1] = tl->u[1] + tl->w[2] * c->r[0] - tl->w[0] * c->r[2];
    c->vco[2] = tl->u[2] + tl->w[0] * c->r[1] - tl->w[1] * c->r[0];
    c->vn = 0.0;
    for (int a = 0; a < 3; ++a) { c->vrel[a] = v[a] - c->vco[a]; c->vn += c->vrel[a] * c->nw[a]; }  /* Eq. 15-16 */
    c->projected = 0;
    c->vtn = 0.0;
    c->s = 0.0;
    c->scale = 1.0;
    if (c->vn < 0.0) {
        c->projected = 1;
        for (int a = 0; a < 3; ++a) { c->vt[a] = c->vrel[a] - c->vn * c->nw[a]; c->vtn += c->vt[a] * c->vt[a]; }  /* Eq. 17 */
        c->vtn = sqrt(c->vtn);
        c->scale = 0.0;             /* Eq. 18, clamped */
        if (c->vtn > 0.0) {
            c->s = c->vtn + p->friction * c->vn;
            c->scale = c->s > 0.0 ? c->s / c->vtn : 0.0;
        }
        for (int a = 0; a < 3; ++a) v[a] = c->scale * c->vt[a] + c->vco[a];  /* Eq. 19 */
    }
}

static inline int in_wall_band(const orc_params *p, int i, int j, int k)
{
    const int b = p->bound, n = p->n_grid;
    return i < b || j < b || k < b || i >= n - b || j >= n - b || k >= n - b;
}

/* grid_v: n^3 x 3 output.  contact (optional, n^3): index of the tool whose
 * projection was applied, -1 otherwise.  margin (optional, n^3): distance of
 * this node's floating-point decisions from a branch point -- min over
 * |d - theta|, |v_n| (if in contact), the gap to the second-closest tool and
 * the distance of x_ref from a cell face of a sampled field (where the
 * sample is within 2h of theta); +inf where no decision depends on the tool. */
void orc_grid_update(const orc_params *p, const orc_tool *tools, int32_t ntools,
                     const double *grid_m, const double *grid_mv, double *grid_v,
                     int32_t *contact, double *margin)
{
    const int n = p->n_grid;
    const double dx = 1.0 / n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                const int64_t I = node_index(n, i, j, k);
                double v[3] = {0.0, 0.0, 0.0};
                int32_t hit = -1;
                double mg = INFINITY;
                if (grid_m[I] > 0.0) {
                    for (int a = 0; a < 3; ++a)
                        v[a] = grid_mv[3 * I + a] / grid_m[I] + p->dt * p->gravity[a];  /* Eq. 7 + gravity */
                    if (ntools > 0) {
                        const double xw[3] = {i * dx, j * dx, k * dx};
                        double nref[3], xref[3], d2, cells;
                        int id;
                        const double dmin = nearest_tool(tools, ntools, p->theta, xw, &id, nref, xref, &d2, &cells);
                        mg = dmin < INFINITY ? fabs(dmin - p->theta) : INFINITY;
                        if (d2 < INFINITY && d2 - dmin < mg) mg = d2 - dmin;
                        if (cells < mg) mg = cells;
                        if (dmin < p->theta) {
                            orc_contact c;
                            contact_response(p, tools + id, xw, nref, v, &c);
                            if (fabs(c.vn) < mg) mg = fabs(c.vn);
                            if (c.projected && c.vtn > 0.0 && fabs(c.s) < mg) mg = fabs(c.s);
                            hit = id;
                        }
                    }
                    if (in_wall_band(p, i, j, k)) {
                        v[0] = v[1] = v[2] = 0.0;          /* sticky walls */
                        mg = INFINITY;
                        hit = -1;
                    }
                }
                for (int a = 0; a < 3; ++a) grid_v[3 * I + a] = v[a];
                if (contact) contact[I] = hit;
                if (margin) margin[I] = mg;
            }
}

/* ---------------------------------------------------- G2P (Eq. 4, 8-10) */

/* Gather grid velocities back to the particles and advect them; updates
 * x, v, C, F in place. */
void orc_g2p(const orc_params *p, const double *grid_v, int64_t N, double *x,
             double *v, double *C, double *F, orc_counters *cnt)
{
    const int n = p->n_grid;
    const double dx = 1.0 / n;
    for (int64_t q = 0; q < N; ++q) {
        double *xp = x + 3 * q, *vp = v + 3 * q, *Cp = C + 9 * q, *Fp = F + 9 * q;
        int base[3];
        double fx[3], w[3][3];
        if (stencil_base(p, xp, base, fx) && cnt) cnt->out_of_domain++;
        for (int d = 0; d < 3; ++d) orc_weights(fx[d], w[d]);
        double vnew[3] = {0, 0, 0}, B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const double wip = w[0][i] * w[1][j] * w[2][k];
                    const double xi_xp[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (k - fx[2]) * dx};
                    const int64_t I = node_index(n, base[0] + i, base[1] + j, base[2] + k);
                    const double *vi = grid_v + 3 * I;
                    for (int a = 0; a < 3; ++a) {
                        vnew[a] += wip * vi[a];                         /* Eq. 8 */
                        for (int b = 0; b < 3; ++b) B[3 * a + b] += wip * vi[a] * xi_xp[b];
                    }
                }
        for (int a = 0; a < 9; ++a) Cp[a] = 4.0 / (dx * dx) * B[a];     /* Eq. 9 */
        double IdtC[9], Fn[9];
        for (int a = 0; a < 9; ++a) IdtC[a] = ((a % 4 == 0) ? 1.0 : 0.0) + p->dt * Cp[a];
        mat_mul(IdtC, Fp, Fn);                                          /* Eq. 4 */
        memcpy(Fp, Fn, sizeof Fn);
        for (int a = 0; a < 3; ++a) {
            vp[a] = vnew[a];
            xp[a] += p->dt * vnew[a];                                   /* Eq. 10 */
        }
    }
}

/* ------------------------------------------------------------- full step */

/* One sub-step: P2G, grid operation, G2P.  scratch must hold 7 n^3 doubles.
 * tools: ntools frames for this sub-step. */
void orc_step(const orc_params *p, const orc_tool *tools, int32_t ntools, int64_t N,
              double *x, double *v, double *C, double *F, double *scratch,
              orc_counters *cnt)
{
    const int64_t nn = (int64_t)p->n_grid * p->n_grid * p->n_grid;
    double *gm = scratch, *gmv = scratch + nn, *gv = scratch + 4 * nn;
    orc_p2g(p, N, x, v, C, F, gm, gmv, cnt);
    orc_grid_update(p, tools, ntools, gm, gmv, gv, NULL, NULL);
    orc_g2p(p, gv, N, x, v, C, F, cnt);
}

/* nsteps sub-steps; tools holds nsteps * ntools frames (sub-step major). */
void orc_run(const orc_params *p, const orc_tool *tools, int32_t ntools, int32_t nsteps,
             int64_t N, double *x, double *v, double *C, double *F, orc_counters *cnt)
{
    const int64_t nn = (int64_t)p->n_grid * p->n_grid * p->n_grid;
    double *scratch = (double *)malloc(sizeof(double) * 7 * nn);
    if (!scratch) return;
    for (int s = 0; s < nsteps; ++s)
        orc_step(p, tools + (int64_t)s * ntools, ntools, N, x, v, C, F, scratch, cnt);
    free(scratch);
}

/* Grid-block key of each particle: the linear index (x fastest) of the
 * 4x4x4-cell block containing base = floor(x/dx - 0.5), computed from the
 * FP32 positions the GPU holds.  Domain clamping as in the stencil. */
void orc_block_keys(int32_t n_grid, int64_t N, const float *x, uint32_t *keys)
{
    const int nb = n_grid / 4;
    for (int64_t q = 0; q < N; ++q) {
        int b[3];
        for (int d = 0; d < 3; ++d) {
            int c = (int)floor((double)x[3 * q + d] * (double)n_grid - 0.5);
            if (c < 0) c = 0;
            if (c > n_grid - 3) c = n_grid - 3;
            b[d] = c / 4;
        }
        keys[q] = (uint32_t)(b[0] + nb * (b[1] + nb * b[2]));
    }
}

/* ======================================================================
 * Adjoint (reverse mode) of one sub-step.
 *
 * The paper does not differentiate its simulator (Sec. V names
 * differentiable physics as future work); this is the plain derivative of
 * orc_step, stage by stage in reverse order (G2P, grid operation, P2G),
 * taken from the formulas above.  Every branch of the forward pass (m > 0,
 * contact d < theta, approaching v_n < 0, the friction clamp, the z-buffer
 * choice, walls, the stencil base) is held at the side the forward pass
 * took, so the result is the derivative of the branch taken.  The distance
 * d only selects branches and contributes no derivative; the sampled field
 * is piecewise constant in x_ref and contributes none either.
 * ====================================================================== */

/* d w / d fx of orc_weights */
static void weights_d(double fx, double *dw)
{
    dw[0] = -(1.5 - fx);
    dw[1] = -2.0 * (fx - 1.0);
    dw[2] = fx - 0.5;
}

/* Jacobian d n / d p (row-major: row = component of n) of the unit normal
 * orc_sdf returns for analytic shapes; zero where that normal is constant
 * (inside a box, on the capsule axis) and for sampled fields. */
static void sdf_normal_jacobian(int32_t kind, const double *dims, const double *p, double *Jn)
{
    for (int i = 0; i < 9; ++i) Jn[i] = 0.0;
    if (kind == 0) {
        double c = p[1];
        int side = 1;                   /* the closest axis point moves with p_y */
        if (c > dims[1]) { c = dims[1]; side = 0; }
        if (c < -dims[1]) { c = -dims[1]; side = 0; }
        const double q[3] = {p[0], p[1] - c, p[2]};
        const double L = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (!(L > 0.0)) return;
        const double u[3] = {q[0] / L, q[1] / L, q[2] / L};
        const double D[3] = {1.0, side ? 0.0 : 1.0, 1.0};   /* d q / d p */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Jn[3 * a + b] = ((a == b ? 1.0 : 0.0) - u[a] * u[b]) / L * D[b];
        return;
    }
    if (kind == 1) {
        double q[3], o[3], s[3], on = 0.0;
        for (int d = 0; d < 3; ++d) {
            q[d] = fabs(p[d]) - dims[d];
            o[d] = q[d] > 0.0 ? q[d] : 0.0;
            s[d] = p[d] < 0.0 ? -1.0 : 1.0;
            on += o[d] * o[d];
        }
        on = sqrt(on);
        if (!(on > 0.0)) return;
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e)
                if (q[d] > 0.0 && q[e] > 0.0)
                    Jn[3 * d + e] = s[d] * s[e] * ((d == e ? 1.0 : 0.0) - o[d] * o[e] / (on * on)) / on;
    }
}

/* Eq. 6 backwards: (dL/dmu, dL/dlam) -> (dL/dE, dL/dnu). */
void orc_lame_vjp(double E, double nu, double mu_bar, double lam_bar, double *E_bar, double *nu_bar)
{
    const double D = (1.0 + nu) * (1.0 - 2.0 * nu);
    *E_bar = mu_bar / (2.0 * (1.0 + nu)) + lam_bar * nu / D;
    *nu_bar = -mu_bar * E / (2.0 * (1.0 + nu) * (1.0 + nu)) + lam_bar * E * (1.0 + 2.0 * nu * nu) / (D * D);
}

/* Reverse mode of orc_step.  x, v, C, F: the state at the START of the
 * sub-step (left unchanged).  xb, vb, Cb, Fb: on entry the adjoint dL/d(state
 * after the sub-step), on return dL/d(state before it).  lame_bar[2]
 * accumulates dL/dmu, dL/dlam; tool_bar (ntools x 18: R row-major, T, u, w
 * of each frame) accumulates dL/d(frame entries).  Returns -1 if scratch
 * memory could not be allocated, else 0. */
/* grid_m, grid_mv: if not NULL, the grid (mass, momentum) the sub-step's
 * grid operation reads, in place of the P2G of (x, v, C, F); the reverse of
 * P2G still differentiates the P2G of the particles.  This evaluates the
 * grid operation and G2P, and their derivatives, at a grid computed
 * elsewhere (in another precision). */
static int step_adjoint_impl(const orc_params *p, const orc_tool *tools, int32_t ntools, int64_t N,
                             const double *x, const double *v, const double *C, const double *F,
                             const double *grid_m, const double *grid_mv,
                             double *xb, double *vb, double *Cb, double *Fb,
                             double *lame_bar, double *tool_bar)
{
    const int n = p->n_grid;
    const double dx = 1.0 / n, K = 4.0 / (dx * dx), dt = p->dt;
    const int64_t nn = (int64_t)n * n * n;
    const double mp = p->rho * p->V0;
    double mu, lam;
    orc_lame(p->E, p->nu, &mu, &lam);
    double *gm = (double *)malloc(sizeof(double) * nn);
    double *gmv = (double *)malloc(sizeof(double) * 3 * nn);
    double *gv = (double *)malloc(sizeof(double) * 3 * nn);
    double *gvb = (double *)calloc(3 * nn, sizeof(double));     /* dL/d(grid velocity) */
    double *gmb = (double *)calloc(nn, sizeof(double));         /* dL/d(grid mass) */
    double *gmvb = (double *)calloc(3 * nn, sizeof(double));    /* dL/d(grid momentum) */
    if (!gm || !gmv || !gv || !gvb || !gmb || !gmvb) {
        free(gm); free(gmv); free(gv); free(gvb); free(gmb); free(gmvb);
        return -1;
    }
    /* the forward pass up to the grid velocities */
    if (grid_m && grid_mv) {
        memcpy(gm, grid_m, sizeof(double) * nn);
        memcpy(gmv, grid_mv, sizeof(double) * 3 * nn);
    } else {
        orc_p2g(p, N, x, v, C, F, gm, gmv, NULL);
    }
    orc_grid_update(p, tools, ntools, gm, gmv, gv, NULL, NULL);

    /* ---- G2P (Eqs. 4, 8-10) backwards */
    for (int64_t q = 0; q < N; ++q) {
        const double *xp = x + 3 * q, *Fp = F + 9 * q;
        int base[3];
        double fx[3], w[3][3], dw[3][3];
        stencil_base(p, xp, base, fx);
        for (int d = 0; d < 3; ++d) { orc_weights(fx[d], w[d]); weights_d(fx[d], dw[d]); }
        double B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const double wip = w[0][i] * w[1][j] * w[2][k];
                    const double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (k - fx[2]) * dx};
                    const double *vi = gv + 3 * node_index(n, base[0] + i, base[1] + j, base[2] + k);
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) B[3 * a + b] += wip * vi[a] * dpos[b];
                }
        double Cn[9], IdtC[9];
        for (int a = 0; a < 9; ++a) { Cn[a] = K * B[a]; IdtC[a] = ((a % 4 == 0) ? 1.0 : 0.0) + dt * Cn[a]; }
        const double *xbo = xb + 3 * q, *vbo = vb + 3 * q, *Cbo = Cb + 9 * q, *Fbo = Fb + 9 * q;
        double vbt[3], Cbt[9], Fbn[9], xbn[3];
        for (int a = 0; a < 3; ++a) { vbt[a] = vbo[a] + dt * xbo[a]; xbn[a] = xbo[a]; }   /* x' = x + dt v' */
        for (int a = 0; a < 3; ++a)                                                       /* F' = (I + dt C') F */
            for (int b = 0; b < 3; ++b) {
                double sF = 0.0, sC = 0.0;
                for (int c = 0; c < 3; ++c) {
                    sF += IdtC[3 * c + a] * Fbo[3 * c + b];
                    sC += Fbo[3 * a + c] * Fp[3 * b + c];
                }
                Fbn[3 * a + b] = sF;
                Cbt[3 * a + b] = Cbo[3 * a + b] + dt * sC;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const double wip = w[0][i] * w[1][j] * w[2][k];
                    const double gw[3] = {dw[0][i] * w[1][j] * w[2][k] * n, w[0][i] * dw[1][j] * w[2][k] * n,
                                          w[0][i] * w[1][j] * dw[2][k] * n};        /* d w_ip / d x_p */
                    const double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (k - fx[2]) * dx};
                    const int64_t I = node_index(n, base[0] + i, base[1] + j, base[2] + k);
                    const double *vi = gv + 3 * I;
                    double s = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double cd = 0.0;
                        for (int b = 0; b < 3; ++b) cd += Cbt[3 * a + b] * dpos[b];
                        gvb[3 * I + a] += wip * (vbt[a] + K * cd);                /* Eqs. 8-9 */
                        s += vi[a] * (vbt[a] + K * cd);
                    }
                    for (int d = 0; d < 3; ++d) xbn[d] += gw[d] * s;
                    for (int b = 0; b < 3; ++b) {                                  /* d dpos / d x_p = -I */
                        double cv = 0.0;
                        for (int a = 0; a < 3; ++a) cv += Cbt[3 * a + b] * vi[a];
                        xbn[b] -= K * wip * cv;
                    }
                }
        for (int a = 0; a < 3; ++a) { xb[3 * q + a] = xbn[a]; vb[3 * q + a] = 0.0; }
        for (int a = 0; a < 9; ++a) { Fb[9 * q + a] = Fbn[a]; Cb[9 * q + a] = 0.0; }
    }

    /* ---- grid operation (Eq. 7, gravity, Eqs. 11-19, walls) backwards */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                const int64_t I = node_index(n, i, j, k);
                if (!(gm[I] > 0.0)) continue;                      /* v = 0: no dependence */
                if (in_wall_band(p, i, j, k)) continue;
                double vf[3], vbar[3];
                for (int a = 0; a < 3; ++a) {
                    vf[a] = gmv[3 * I + a] / gm[I] + dt * p->gravity[a];
                    vbar[a] = gvb[3 * I + a];
                }
                if (ntools > 0) {
                    const double xw[3] = {i * dx, j * dx, k * dx};
                    double nref[3], xref[3], d2;
                    int id;
                    const double dmin = nearest_tool(tools, ntools, p->theta, xw, &id, nref, xref, &d2, NULL);
                    if (dmin < p->theta) {
                        const orc_tool *tl = tools + id;
                        double vout[3] = {vf[0], vf[1], vf[2]};
                        orc_contact c;
                        contact_response(p, tl, xw, nref, vout, &c);
                        if (c.projected) {
                            /* v' = scale vt + vco */
                            double vtb[3] = {0, 0, 0}, vnb = 0.0, nwb[3], vrelb[3], vcob[3];
                            if (c.scale > 0.0) {
                                double scb = 0.0;
                                for (int a = 0; a < 3; ++a) { vtb[a] = c.scale * vbar[a]; scb += vbar[a] * c.vt[a]; }
                                /* scale = 1 + mu_f vn / |vt| */
                                vnb += p->friction * scb / c.vtn;
                                const double vtnb = -p->friction * c.vn * scb / (c.vtn * c.vtn);
                                for (int a = 0; a < 3; ++a) vtb[a] += vtnb * c.vt[a] / c.vtn;
                            }
                            /* vt = vrel - vn nw */
                            double vtb_n = 0.0;
                            for (int a = 0; a < 3; ++a) { vrelb[a] = vtb[a]; vtb_n += vtb[a] * c.nw[a]; nwb[a] = -c.vn * vtb[a]; }
                            vnb -= vtb_n;
                            /* vn = vrel . nw */
                            for (int a = 0; a < 3; ++a) { vrelb[a] += vnb * c.nw[a]; nwb[a] += vnb * c.vrel[a]; }
                            /* vrel = v - vco, and v' carries + vco */
                            for (int a = 0; a < 3; ++a) vcob[a] = vbar[a] - vrelb[a];
                            double *tb = tool_bar + 18 * id;           /* R[9], T[3], u[3], w[3] */
                            /* vco = u + w x r, r = x - T */
                            double rb[3];
                            for (int a = 0; a < 3; ++a) tb[12 + a] += vcob[a];
                            tb[15] += c.r[1] * vcob[2] - c.r[2] * vcob[1];
                            tb[16] += c.r[2] * vcob[0] - c.r[0] * vcob[2];
                            tb[17] += c.r[0] * vcob[1] - c.r[1] * vcob[0];
                            rb[0] = vcob[1] * tl->w[2] - vcob[2] * tl->w[1];
                            rb[1] = vcob[2] * tl->w[0] - vcob[0] * tl->w[2];
                            rb[2] = vcob[0] * tl->w[1] - vcob[1] * tl->w[0];
                            for (int a = 0; a < 3; ++a) tb[9 + a] -= rb[a];
                            /* nw = R nref(x_ref), x_ref = R^T (x - T) */
                            double nrb[3], Jn[9], xrb[3];
                            for (int a = 0; a < 3; ++a)
                                for (int e = 0; e < 3; ++e) tb[3 * a + e] += nwb[a] * nref[e];
                            for (int e = 0; e < 3; ++e) {
                                nrb[e] = 0.0;
                                for (int a = 0; a < 3; ++a) nrb[e] += tl->R[3 * a + e] * nwb[a];
                            }
                            if (tl->kind != 2) sdf_normal_jacobian(tl->kind, tl->dims, xref, Jn);
                            else for (int a = 0; a < 9; ++a) Jn[a] = 0.0;
                            for (int e = 0; e < 3; ++e) {
                                xrb[e] = 0.0;
                                for (int a = 0; a < 3; ++a) xrb[e] += Jn[3 * a + e] * nrb[a];
                            }
                            for (int e = 0; e < 3; ++e)
                                for (int a = 0; a < 3; ++a) tb[3 * e + a] += c.r[e] * xrb[a];
                            for (int e = 0; e < 3; ++e) {
                                double s = 0.0;
                                for (int a = 0; a < 3; ++a) s += tl->R[3 * e + a] * xrb[a];
                                tb[9 + e] -= s;
                            }
                            for (int a = 0; a < 3; ++a) vbar[a] = vrelb[a];
                        }
                    }
                }
                /* v = mv / m + dt g */
                double dotv = 0.0;
                for (int a = 0; a < 3; ++a) {
                    gmvb[3 * I + a] = vbar[a] / gm[I];
                    dotv += vbar[a] * gmv[3 * I + a];
                }
                gmb[I] = -dotv / (gm[I] * gm[I]);
            }

    /* ---- P2G (Eqs. 1-3, 5-6) backwards */
    for (int64_t q = 0; q < N; ++q) {
        const double *xp = x + 3 * q, *vp = v + 3 * q, *Cp = C + 9 * q, *Fp = F + 9 * q;
        int base[3];
        double fx[3], w[3][3], dw[3][3];
        stencil_base(p, xp, base, fx);
        for (int d = 0; d < 3; ++d) { orc_weights(fx[d], w[d]); weights_d(fx[d], dw[d]); }
        double tau[9], A[9];
        orc_piola_FT(mu, lam, Fp, tau);
        for (int a = 0; a < 9; ++a) A[a] = mp * Cp[a] - dt * K * p->V0 * tau[a];
        double Ab[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, vbp[3] = {0, 0, 0}, xbp[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const double wip = w[0][i] * w[1][j] * w[2][k];
                    const double gw[3] = {dw[0][i] * w[1][j] * w[2][k] * n, w[0][i] * dw[1][j] * w[2][k] * n,
                                          w[0][i] * w[1][j] * dw[2][k] * n};
                    const double dpos[3] = {(i - fx[0]) * dx, (j - fx[1]) * dx, (k - fx[2]) * dx};
                    const int64_t I = node_index(n, base[0] + i, base[1] + j, base[2] + k);
                    const double *mvb = gmvb + 3 * I;
                    double s = gmb[I] * mp;
                    for (int a = 0; a < 3; ++a) {
                        double mom = mp * vp[a];
                        for (int b = 0; b < 3; ++b) {
                            mom += A[3 * a + b] * dpos[b];
                            Ab[3 * a + b] += wip * mvb[a] * dpos[b];
                        }
                        s += mvb[a] * mom;
                        vbp[a] += mp * wip * mvb[a];
                    }
                    for (int d = 0; d < 3; ++d) xbp[d] += gw[d] * s;
                    for (int b = 0; b < 3; ++b) {
                        double am = 0.0;
                        for (int a = 0; a < 3; ++a) am += A[3 * a + b] * mvb[a];
                        xbp[b] -= wip * am;
                    }
                }
        /* A = m C - dt (4/dx^2) V0 tau,  tau = mu (F F^T - I) + lam ln(J) I */
        double taub[9], trb = 0.0;
        for (int a = 0; a < 9; ++a) { Cb[9 * q + a] = mp * Ab[a]; taub[a] = -dt * K * p->V0 * Ab[a]; }
        trb = taub[0] + taub[4] + taub[8];
        const double J = mat_det(Fp);
        double FFt[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += Fp[3 * a + c] * Fp[3 * b + c];
                FFt[3 * a + b] = s - (a == b ? 1.0 : 0.0);
            }
        double mub = 0.0;
        for (int a = 0; a < 9; ++a) mub += taub[a] * FFt[a];
        lame_bar[0] += mub;
        lame_bar[1] += trb * (J > 0.0 ? log(J) : log(1e-6));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int c = 0; c < 3; ++c) s += (taub[3 * a + c] + taub[3 * c + a]) * Fp[3 * c + b];
                Fb[9 * q + 3 * a + b] += mu * s;
            }
        if (J > 0.0) {
            double FiT[9];
            mat_inv_transpose(Fp, J, FiT);
            for (int a = 0; a < 9; ++a) Fb[9 * q + a] += lam * trb * FiT[a];
        }
        for (int a = 0; a < 3; ++a) { vb[3 * q + a] = vbp[a]; xb[3 * q + a] += xbp[a]; }
    }
    free(gm); free(gmv); free(gv); free(gvb); free(gmb); free(gmvb);
    return 0;
}

int orc_step_adjoint(const orc_params *p, const orc_tool *tools, int32_t ntools, int64_t N,
                     const double *x, const double *v, const double *C, const double *F,
                     double *xb, double *vb, double *Cb, double *Fb,
                     double *lame_bar, double *tool_bar)
{
    return step_adjoint_impl(p, tools, ntools, N, x, v, C, F, NULL, NULL, xb, vb, Cb, Fb, lame_bar, tool_bar);
}

int orc_step_adjoint_at_grid(const orc_params *p, const orc_tool *tools, int32_t ntools, int64_t N,
                             const double *x, const double *v, const double *C, const double *F,
                             const double *grid_m, const double *grid_mv,
                             double *xb, double *vb, double *Cb, double *Fb,
                             double *lame_bar, double *tool_bar)
{
    return step_adjoint_impl(p, tools, ntools, N, x, v, C, F, grid_m, grid_mv, xb, vb, Cb, Fb, lame_bar,
                             tool_bar);
}

/* ======================================================================
 * Surface extraction (the renderer's Marching Cubes step of Sec. III).
 *
 * The iso-surface field >= iso of a node field is triangulated cell by
 * cell.  Each cell is split into six tetrahedra around its diagonal from
 * corner 0 to corner 7 (corner c sits at offset (c & 1, (c >> 1) & 1,
 * (c >> 2) & 1)); every tetrahedron contributes 0, 1 or 2 triangles, and
 * neighbouring cells split their shared faces alike, so the surface is
 * closed.  Vertices lie on tetrahedron edges at the linear interpolation
 * of the field, computed from the lower-numbered corner; triangles face
 * away from the inside (field >= iso).  This reading avoids the ambiguous
 * faces of the 256-case cube table.
 * ====================================================================== */

static const int orc_tet_paths[6][2] = {{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}};

static void corner_offset(int c, int *o)
{
    o[0] = c & 1; o[1] = (c >> 1) & 1; o[2] = (c >> 2) & 1;
}

/* sign of det[B - A, C - A, D - A] for cube corners A..D (exact integers) */
static int tet_orientation(int a, int b, int c, int d)
{
    int pa[3], pb[3], pc[3], pd[3];
    corner_offset(a, pa); corner_offset(b, pb); corner_offset(c, pc); corner_offset(d, pd);
    const int u[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
    const int v[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
    const int w[3] = {pd[0] - pa[0], pd[1] - pa[1], pd[2] - pa[2]};
    const int det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) + u[2] * (v[0] * w[1] - v[1] * w[0]);
    return det > 0 ? 1 : -1;
}

/* point where the field crosses iso on the edge between cube corners a, b */
static void edge_point(const int *cell, int a, int b, const double *f, double iso, double dx, double *out)
{
    if (a > b) { const int t = a; a = b; b = t; }
    int pa[3], pb[3];
    corner_offset(a, pa);
    corner_offset(b, pb);
    const double t = (iso - f[a]) / (f[b] - f[a]);
    for (int d = 0; d < 3; ++d)
        out[d] = ((double)(cell[d] + pa[d]) + t * (double)(pb[d] - pa[d])) * dx;
}

static int64_t emit(double *out, int64_t cnt, int64_t max_tri, const int *cell, const double *f, double iso,
                    double dx, const int e[3][2])
{
    if (cnt < max_tri && out)
        for (int v = 0; v < 3; ++v) edge_point(cell, e[v][0], e[v][1], f, iso, dx, out + 9 * cnt + 3 * v);
    return cnt + 1;
}

/* Triangles of one tetrahedron (corners t[4] positively oriented). */
static int64_t tet_triangles(const int *cell, const int *t, const double *f, double iso, double dx, double *out,
                             int64_t cnt, int64_t max_tri)
{
    int in[4], nin = 0;
    for (int q = 0; q < 4; ++q) { in[q] = f[t[q]] >= iso; nin += in[q]; }
    if (nin == 0 || nin == 4) return cnt;
    if (nin == 1 || nin == 3) {
        /* the lone vertex (inside for nin = 1, outside for nin = 3) first, in
           an even permutation of t */
        int lone = 0;
        for (int q = 0; q < 4; ++q) if (in[q] == (nin == 1)) lone = q;
        static const int even_first[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 0, 1, 3}, {3, 0, 2, 1}};
        const int *p = even_first[lone];
        int e[3][2] = {{t[p[0]], t[p[1]]}, {t[p[0]], t[p[2]]}, {t[p[0]], t[p[3]]}};
        if (nin == 3) { int s0 = e[1][0], s1 = e[1][1]; e[1][0] = e[2][0]; e[1][1] = e[2][1]; e[2][0] = s0; e[2][1] = s1; }
        return emit(out, cnt, max_tri, cell, f, iso, dx, e);
    }
    /* two inside (p, q) and two outside (r, s), (p, q, r, s) an even permutation */
    int ins[2], outs[2], a = 0, b = 0;
    for (int k = 0; k < 4; ++k) { if (in[k]) ins[a++] = k; else outs[b++] = k; }
    int perm[4] = {ins[0], ins[1], outs[0], outs[1]};
    int inv = 0;                                  /* parity of perm */
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) inv += perm[i] > perm[j];
    if (inv & 1) { const int x = perm[2]; perm[2] = perm[3]; perm[3] = x; }
    const int P = t[perm[0]], Q = t[perm[1]], R = t[perm[2]], S = t[perm[3]];
    const int e1[3][2] = {{P, R}, {P, S}, {Q, S}};
    const int e2[3][2] = {{P, R}, {Q, S}, {Q, R}};
    cnt = emit(out, cnt, max_tri, cell, f, iso, dx, e1);
    return emit(out, cnt, max_tri, cell, f, iso, dx, e2);
}

/* field: n^3 node values, [i][j][k] with k fastest; node (i, j, k) sits at
 * (i, j, k) dx.  Writes up to max_tri triangles (9 doubles each: three
 * vertices) in cell order with i fastest, then j, then k, tetrahedra in the
 * order of orc_tet_paths; returns the total number of triangles. */
int64_t orc_surface(int32_t n, const double *field, double iso, double dx, double *out, int64_t max_tri)
{
    int64_t cnt = 0;
    for (int k = 0; k + 1 < n; ++k)
        for (int j = 0; j + 1 < n; ++j)
            for (int i = 0; i + 1 < n; ++i) {
                const int cell[3] = {i, j, k};
                double f[8];
                for (int c = 0; c < 8; ++c) {
                    int o[3];
                    corner_offset(c, o);
                    f[c] = field[node_index(n, i + o[0], j + o[1], k + o[2])];
                }
                for (int q = 0; q < 6; ++q) {
                    int t[4] = {0, orc_tet_paths[q][0], orc_tet_paths[q][1], 7};
                    if (tet_orientation(t[0], t[1], t[2], t[3]) < 0) { const int x = t[1]; t[1] = t[2]; t[2] = x; }
                    cnt = tet_triangles(cell, t, f, iso, dx, out, cnt, max_tri);
                }
            }
    return cnt;
}
