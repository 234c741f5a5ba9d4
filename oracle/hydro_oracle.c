/*
 * hydro_oracle.c -- plain, slow FP64 CPU oracle for the relaxing-TVD
 * patch-group hydro path of GAMER (Schive, Tsai & Chiueh, arXiv 0907.3390).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library; it is compiled with
 * -ffp-contract=off so that every operation below rounds once, in the order
 * written.
 *
 * What it computes (paper sections):
 *   - ideal-gas Euler equations in conservative form, u = (rho, rho v, e)
 *     (Sec. 2.2, Eqs. MassConserve..EnergyConserve, ThermalEnergy, EOS);
 *   - the 1-D relaxing TVD scheme: freezing speed c = |v| + c_s, right/left
 *     moving fluxes F^R, F^L (Eq. LRFlux), first-order upwind half step
 *     (Eq. MidpointValue), second-order TVD full step with the van Leer
 *     limiter (Eqs. 2ndTVDFluxCorr, 2ndFluxCorr, vanLeer, 2ndRFlux,
 *     FullstepValue); minmod is offered as an alternative limiter;
 *   - Strang dimensional splitting, forward sweep xyz / backward sweep zyx
 *     with the same dt (Sec. 2.2, last paragraphs);
 *   - patch groups of 2x2x2 patches of 8^3 cells padded by 3 ghost cells,
 *     ghost cells copied from same-level neighbours or interpolated with the
 *     Min-Mod limiter from the level one coarser (Sec. 2.2, Sec. 3.1);
 *   - restriction (coarse = mean of 8 children) and coarse-fine flux
 *     correction (Sec. 2.1, step 3 of the level evolution);
 *   - the CFL time step (Sec. 3.4, Eq. CFL);
 *   - conservation sums and a positivity count over leaf cells.
 *
 * Readings where the paper is silent or loose (each one listed in the design
 * notes of the repository):
 *   R1 one call = one sweep set (xyz when order = 0, zyx when order = 1);
 *   R2 the freezing speed is per cell, |v_normal| + c_s;
 *   R3 F^R = (c u + F)/2 and F^L = (c u - F)/2, i.e. c (u +- w)/2 with
 *      w = F/c substituted; w itself is never formed;
 *   R4 the left-moving TVD flux mirrors Eq. 2ndRFlux with upwind cell n+1;
 *   R5 van Leer is applied only when the product of the two corrections is
 *      strictly positive; minmod likewise;
 *   R6 c_s uses max(P, 0); conserved variables are never floored;
 *   R7 coarse data used for fine ghost cells is the pre-step coarse state;
 *   R8 Min-Mod interpolation acts on conserved variables, one slope per axis
 *      from the two face neighbours of the coarse cell, child value
 *      U_C + ((sx*Sx + sy*Sy) + sz*Sz)/4 with s* = -1 for the lower child;
 *   R9 a uniform dt for all levels.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NV 5      /* conserved variables rho, mx, my, mz, e          */
#define PS 8      /* patch size (cells per axis)                      */
#define GS 16     /* patch-group size (2 patches per axis)            */
#define NG 3      /* ghost cells per side (seven-point stencil)       */
#define PD 22     /* padded patch-group size GS + 2*NG                */

enum { ORC_VANLEER = 0, ORC_MINMOD = 1 };
#define MAXLV 16
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_MAP = -3 };

/* One refinement level as the oracle sees it.  All arrays are host memory.
 * u / u_out: [NV][8*n_groups][8][8][8] (x fastest); nbr: [n_groups][26];
 * parent: [n_groups] (patch index on the level below, NULL on level 0);
 * child: [8*n_groups] (patch-group index on the level above or -1, NULL if
 * there is no finer level); face_flux: [n_groups][3][3][NV][16][16] or NULL. */
typedef struct {
    int32_t n_groups;
    int32_t pad_;
    double dh;
    const double *u;
    double *u_out;
    const int32_t *nbr;
    const int32_t *parent;
    const int32_t *child;
    double *face_flux;
    /* individual time steps (Sec. 2.1): */
    const double *u_new;    /* this level's state after its current sweep set,
                               read by the finer level's coarse ghosts; NULL: none */
    double coarse_w;        /* weight of the coarser level's u_new in this level's
                               coarse ghosts (0 for the first of its two steps,
                               1/2 for the second) */
    double *face_flux2;     /* this level's face fluxes of its second step; with
                               face_flux (first step) averaged by the coarser
                               level's fix-up; NULL: one step per coarse step */
} orc_level;

/* ---------------------------------------------------------------- limiters */

/* Eq. vanLeer: harmonic combination of the two second-order corrections. */
double orc_phi_vanleer(double a, double b)
{
    if (a * b > 0.0)
        return 2.0 * a * b / (a + b);
    return 0.0;
}

/* minmod: the smaller correction in magnitude when both have one sign. */
double orc_phi_minmod(double a, double b)
{
    if (a * b > 0.0) {
        double m = fmin(fabs(a), fabs(b));
        return a > 0.0 ? m : -m;
    }
    return 0.0;
}

static double phi(int limiter, double a, double b)
{
    return limiter == ORC_MINMOD ? orc_phi_minmod(a, b) : orc_phi_vanleer(a, b);
}

/* ------------------------------------------------- cell state and fluxes */

/* Pressure from Eqs. ThermalEnergy and EOS: P = (gamma-1)(e - rho v^2 / 2). */
double orc_pressure(const double u[NV], double gamma)
{
    double rho = u[0];
    double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
    double eps = u[4] - 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    return (gamma - 1.0) * eps;
}

/* Right- and left-moving fluxes of one cell for a sweep along axis d
 * (Eq. LRFlux with the freezing speed c = |v_d| + c_s of Sec. 2.2). */
static void cell_lr_flux(const double u[NV], int d, double gamma,
                         double FR[NV], double FL[NV])
{
    double rho = u[0];
    double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
    double eps = u[4] - 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    double P = (gamma - 1.0) * eps;
    double cs = sqrt(gamma * fmax(P, 0.0) / rho);
    double vn = d == 0 ? vx : (d == 1 ? vy : vz);
    double c = fabs(vn) + cs;
    double F[NV];
    /* F = (rho v_d, rho v v_d + P delta, (e + P) v_d) */
    F[0] = u[1 + d];
    F[1] = u[1] * vn;
    F[2] = u[2] * vn;
    F[3] = u[3] * vn;
    F[1 + d] = u[1 + d] * vn + P;
    F[4] = (u[4] + P) * vn;
    for (int v = 0; v < NV; v++) {
        FR[v] = 0.5 * (c * u[v] + F[v]);
        FL[v] = 0.5 * (c * u[v] - F[v]);
    }
}

/* One relaxing-TVD step of a 1-D column q[0..L-1] along axis d
 * (Eqs. MidpointValue, 2ndTVDFluxCorr, 2ndFluxCorr, 2ndRFlux,
 * FullstepValue).  Cells 3..L-4 of out[] receive the full-step values; the
 * net interface fluxes G[n] of interface n+1/2 (n = 2..L-4) are returned in
 * G when it is not NULL. */
static void tvd_column(const double (*q)[NV], int L, int d, double lam,
                       double gamma, int limiter, double (*out)[NV],
                       double (*G)[NV])
{
    double (*FR)[NV] = malloc(sizeof(double) * NV * L);
    double (*FL)[NV] = malloc(sizeof(double) * NV * L);
    double (*Fh)[NV] = malloc(sizeof(double) * NV * L);
    double (*uh)[NV] = malloc(sizeof(double) * NV * L);
    double (*Gl)[NV] = malloc(sizeof(double) * NV * L);

    /* half step: first-order upwind interface flux F_{n+1/2} = F^R_n - F^L_{n+1} */
    for (int n = 0; n < L; n++)
        cell_lr_flux(q[n], d, gamma, FR[n], FL[n]);
    for (int n = 0; n + 1 < L; n++)
        for (int v = 0; v < NV; v++)
            Fh[n][v] = FR[n][v] - FL[n + 1][v];
    for (int n = 1; n + 1 < L; n++)
        for (int v = 0; v < NV; v++)
            uh[n][v] = q[n][v] - 0.5 * lam * (Fh[n][v] - Fh[n - 1][v]);

    /* full step: TVD fluxes of the midpoint state */
    for (int n = 1; n + 1 < L; n++)
        cell_lr_flux(uh[n], d, gamma, FR[n], FL[n]);
    for (int n = 2; n + 3 < L; n++) {
        for (int v = 0; v < NV; v++) {
            double a = (FR[n][v] - FR[n - 1][v]) / 2.0;
            double b = (FR[n + 1][v] - FR[n][v]) / 2.0;
            double FRh = FR[n][v] + phi(limiter, a, b);
            a = (FL[n + 1][v] - FL[n + 2][v]) / 2.0;
            b = (FL[n][v] - FL[n + 1][v]) / 2.0;
            double FLh = FL[n + 1][v] + phi(limiter, a, b);
            Gl[n][v] = FRh - FLh;
        }
    }
    for (int n = 3; n + 3 < L; n++)
        for (int v = 0; v < NV; v++)
            out[n][v] = q[n][v] - lam * (Gl[n][v] - Gl[n - 1][v]);
    if (G)
        for (int n = 2; n + 3 < L; n++)
            for (int v = 0; v < NV; v++)
                G[n][v] = Gl[n][v];
    free(FR); free(FL); free(Fh); free(uh); free(Gl);
}

/* Exported for the column-level tests: q is [L][NV], out receives [L][NV]
 * with cells 3..L-4 updated (others copied). */
int orc_tvd_column(const double *q, int L, int d, double lam, double gamma,
                   int limiter, double *out)
{
    if (L < 7 || d < 0 || d > 2)
        return ORC_ERR_ARG;
    memcpy(out, q, sizeof(double) * NV * L);
    tvd_column((const double (*)[NV])q, L, d, lam, gamma, limiter,
               (double (*)[NV])out, NULL);
    return ORC_OK;
}

/* ---------------------------------------------- whole-domain split solver */

/* One sweep set (xyz if order == 0, zyx otherwise) on a whole single-level
 * domain u[NV][nz][ny][nx] (x fastest).  bc[a] = 0: periodic along axis a,
 * 1: outflow (zero-gradient).  Every column is padded with 3 ghost cells
 * from its own boundary rule, updated by the 1-D scheme, and written back. */
int orc_domain_sweepset(double *u, int nx, int ny, int nz, const int *bc,
                        double gamma, int limiter, double dt, double dh,
                        int order)
{
    if (nx < 1 || ny < 1 || nz < 1 || dh <= 0.0)
        return ORC_ERR_ARG;
    const int n[3] = {nx, ny, nz};
    const long st[3] = {1, nx, (long)nx * ny};
    const long ncell = (long)nx * ny * nz;
    const double lam = dt / dh;
    for (int s = 0; s < 3; s++) {
        int a = order == 0 ? s : 2 - s;
        int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
        int L = n[a] + 2 * NG;
        long ncol = (long)n[t1] * n[t2];
#pragma omp parallel for schedule(static)
        for (long col = 0; col < ncol; col++) {
            double (*q)[NV] = malloc(sizeof(double) * NV * L);
            double (*o)[NV] = malloc(sizeof(double) * NV * L);
            int i1 = (int)(col % n[t1]), i2 = (int)(col / n[t1]);
            long base = i1 * st[t1] + i2 * st[t2];
            for (int k = 0; k < L; k++) {
                int x = k - NG;
                if (bc[a] == 0)
                    x = ((x % n[a]) + n[a]) % n[a];
                else
                    x = x < 0 ? 0 : (x >= n[a] ? n[a] - 1 : x);
                for (int v = 0; v < NV; v++)
                    q[k][v] = u[v * ncell + base + x * st[a]];
            }
            tvd_column((const double (*)[NV])q, L, a, lam, gamma, limiter, o, NULL);
            for (int k = NG; k < L - NG; k++)
                for (int v = 0; v < NV; v++)
                    u[v * ncell + base + (k - NG) * st[a]] = o[k][v];
            free(q);
            free(o);
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------ patch-group form */

static int dir_index(int dx, int dy, int dz)
{
    int d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    return d < 13 ? d : d - 1;
}

static int floordiv(int a, int b)
{
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0)))
        q--;
    return q;
}

/* Index of cell (x,y,z), 0 <= x,y,z < 16, of patch group g, variable v. */
static size_t cell_index(const orc_level *L, int g, int v, int x, int y, int z)
{
    size_t patch = (size_t)8 * g + (size_t)(((z / PS) * 2 + (y / PS)) * 2 + (x / PS));
    return ((size_t)v * 8 * L->n_groups + patch) * (PS * PS * PS) +
           (size_t)(((z % PS) * PS + (y % PS)) * PS + (x % PS));
}

/* Value of the cell at patch-group-local position (x,y,z) of group g on one
 * level, -16 <= x,y,z < 32.  Axes whose face neighbour is an outflow
 * boundary (-2) are clamped into the group first (zero gradient); the rest
 * are resolved through the neighbour map.  Returns 0 on success, 1 if the
 * position lies in a region that only exists on the coarser level (-1),
 * ORC_ERR_MAP on an inconsistent map. */
static int level_fetch(const orc_level *L, const double *u, int g, int x,
                       int y, int z, double val[NV])
{
    int c[3] = {x, y, z};
    int o[3];
    for (int a = 0; a < 3; a++) {
        o[a] = floordiv(c[a], GS);
        if (o[a] != 0) {
            int e[3] = {0, 0, 0};
            e[a] = o[a];
            if (L->nbr[(size_t)g * 26 + dir_index(e[0], e[1], e[2])] == -2) {
                c[a] = c[a] < 0 ? 0 : GS - 1;
                o[a] = 0;
            }
        }
    }
    int n = g;
    if (o[0] || o[1] || o[2])
        n = L->nbr[(size_t)g * 26 + dir_index(o[0], o[1], o[2])];
    if (n == -1)
        return 1;
    if (n < 0 || n >= L->n_groups)
        return ORC_ERR_MAP;
    for (int v = 0; v < NV; v++)
        val[v] = u[cell_index(L, n, v, c[0] - GS * o[0], c[1] - GS * o[1],
                              c[2] - GS * o[2])];
    return 0;
}

/* Coarse value for the ghosts of the finer level: the coarser level's state
 * before its sweep set, or with individual time steps the linear
 * interpolation in time u + w (u_new - u) to the start of the finer
 * level's step (w = 0 or 1/2). */
static int coarse_fetch(const orc_level *C, double w, int g, int x, int y, int z, double val[NV])
{
    int r = level_fetch(C, C->u, g, x, y, z, val);
    if (r != 0 || w == 0.0 || C->u_new == NULL)
        return r;
    double b[NV];
    r = level_fetch(C, C->u_new, g, x, y, z, b);
    if (r != 0)
        return r;
    for (int v = 0; v < NV; v++)
        val[v] = val[v] + w * (b[v] - val[v]);
    return 0;
}

static double minmod2(double a, double b)
{
    if (a * b > 0.0) {
        double m = fmin(fabs(a), fabs(b));
        return a > 0.0 ? m : -m;
    }
    return 0.0;
}

/* Conservative linear interpolation with the Min-Mod limiter from the level
 * one coarser (Sec. 2.1 refinement step, Sec. 2.2 ghost zones; reading R8).
 * (x,y,z) is a fine position relative to fine group g, the coarse data is
 * the pre-step state of level lv-1 (reading R7), interpolated in time with
 * individual time steps (reading R18). */
static int prolong_fetch(const orc_level *lv, int l, int g, int x, int y, int z,
                         double val[NV])
{
    if (l == 0 || lv[l].parent == NULL)
        return ORC_ERR_MAP;
    const orc_level *C = &lv[l - 1];
    int P = lv[l].parent[g];
    if (P < 0 || P >= 8 * C->n_groups)
        return ORC_ERR_MAP;
    int gc = P / 8, lp = P % 8;
    int pc[3] = {lp & 1, (lp >> 1) & 1, (lp >> 2) & 1};
    int f[3] = {x, y, z};
    int cc[3], sg[3];
    for (int a = 0; a < 3; a++) {
        cc[a] = PS * pc[a] + floordiv(f[a], 2);
        sg[a] = (f[a] - 2 * floordiv(f[a], 2)) == 0 ? -1 : 1;
    }
    double U[NV], Um[NV], Up[NV], S[3][NV];
    const double w = lv[l].coarse_w;
    if (coarse_fetch(C, w, gc, cc[0], cc[1], cc[2], U) != 0)
        return ORC_ERR_MAP;
    for (int a = 0; a < 3; a++) {
        int m[3] = {cc[0], cc[1], cc[2]}, p[3] = {cc[0], cc[1], cc[2]};
        m[a] -= 1;
        p[a] += 1;
        if (coarse_fetch(C, w, gc, m[0], m[1], m[2], Um) != 0 ||
            coarse_fetch(C, w, gc, p[0], p[1], p[2], Up) != 0)
            return ORC_ERR_MAP;
        for (int v = 0; v < NV; v++)
            S[a][v] = minmod2(U[v] - Um[v], Up[v] - U[v]);
    }
    for (int v = 0; v < NV; v++) {
        double t = (sg[0] * S[0][v] + sg[1] * S[1][v]) + sg[2] * S[2][v];
        val[v] = U[v] + 0.25 * t;
    }
    return 0;
}

/* Exported for the interpolation tests: the 8 children of the coarse cell at
 * the centre of a 3x3x3 block c[NV][3][3][3] (x fastest), written to
 * out[NV][2][2][2] (x fastest). */
int orc_minmod_children(const double *c, double *out)
{
    for (int v = 0; v < NV; v++) {
        const double *b = c + v * 27;
        double U = b[13];
        double S[3];
        S[0] = minmod2(U - b[12], b[14] - U);
        S[1] = minmod2(U - b[10], b[16] - U);
        S[2] = minmod2(U - b[4], b[22] - U);
        for (int k = 0; k < 2; k++)
            for (int j = 0; j < 2; j++)
                for (int i = 0; i < 2; i++) {
                    double sx = i ? 1.0 : -1.0, sy = j ? 1.0 : -1.0, sz = k ? 1.0 : -1.0;
                    double t = (sx * S[0] + sy * S[1]) + sz * S[2];
                    out[v * 8 + (k * 2 + j) * 2 + i] = U + 0.25 * t;
                }
    }
    return ORC_OK;
}

/* Build the padded 22^3 block of group g on level l: interior and
 * same-level ghosts copied, coarse ghosts interpolated. blk[NV][22][22][22]. */
static int gather_block(const orc_level *lv, int l, int g, double *blk)
{
    const orc_level *L = &lv[l];
    double val[NV];
    for (int k = 0; k < PD; k++)
        for (int j = 0; j < PD; j++)
            for (int i = 0; i < PD; i++) {
                int r = level_fetch(L, L->u, g, i - NG, j - NG, k - NG, val);
                if (r == 1)
                    r = prolong_fetch(lv, l, g, i - NG, j - NG, k - NG, val);
                if (r != 0)
                    return ORC_ERR_MAP;
                for (int v = 0; v < NV; v++)
                    blk[((size_t)(v * PD + k) * PD + j) * PD + i] = val[v];
            }
    return ORC_OK;
}

/* Advance the listed patch groups of level l by one sweep set (all groups
 * if list == NULL): gather, three sweeps on the shrinking regions of
 * Sec. 3.1 (x on 16x22x22 outputs, y on 16x16x22, z on 16^3 for xyz;
 * mirrored for zyx), write the 16^3 interior to u_out and, when face_flux
 * is given, the net fluxes on the interior-relative planes 0, 8, 16 of each
 * axis for the 16x16 interior rows. */
int orc_level_advance(const orc_level *lv, int n_levels, int l, double gamma,
                      int limiter, double dt, int order, const int32_t *list,
                      int n_list)
{
    if (l < 0 || l >= n_levels)
        return ORC_ERR_ARG;
    const orc_level *L = &lv[l];
    int count = list ? n_list : L->n_groups;
    const double lam = dt / L->dh;
    int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int it = 0; it < count; it++) {
        int g = list ? list[it] : it;
        double *blk = malloc(sizeof(double) * NV * PD * PD * PD);
        double (*q)[NV] = malloc(sizeof(double) * NV * PD);
        double (*o)[NV] = malloc(sizeof(double) * NV * PD);
        double (*G)[NV] = malloc(sizeof(double) * NV * PD);
        if (gather_block(lv, l, g, blk) != ORC_OK) {
#pragma omp critical
            err = ORC_ERR_MAP;
            free(blk); free(q); free(o); free(G);
            continue;
        }
        const long st[3] = {1, PD, PD * PD};
        int swept[3] = {0, 0, 0};
        for (int s = 0; s < 3; s++) {
            int a = order == 0 ? s : 2 - s;
            int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
            int lo1 = swept[t1] ? NG : 0, hi1 = swept[t1] ? NG + GS : PD;
            int lo2 = swept[t2] ? NG : 0, hi2 = swept[t2] ? NG + GS : PD;
            for (int i2 = lo2; i2 < hi2; i2++)
                for (int i1 = lo1; i1 < hi1; i1++) {
                    long base = i1 * st[t1] + i2 * st[t2];
                    for (int k = 0; k < PD; k++)
                        for (int v = 0; v < NV; v++)
                            q[k][v] = blk[(long)v * PD * PD * PD + base + k * st[a]];
                    tvd_column((const double (*)[NV])q, PD, a, lam, gamma, limiter, o, G);
                    for (int k = NG; k < NG + GS; k++)
                        for (int v = 0; v < NV; v++)
                            blk[(long)v * PD * PD * PD + base + k * st[a]] = o[k][v];
                    int interior = i1 >= NG && i1 < NG + GS && i2 >= NG && i2 < NG + GS;
                    if (L->face_flux && interior) {
                        for (int p = 0; p < 3; p++)
                            for (int v = 0; v < NV; v++) {
                                size_t idx = ((((size_t)g * 3 + a) * 3 + p) * NV + v) * GS * GS +
                                             (size_t)(i2 - NG) * GS + (i1 - NG);
                                L->face_flux[idx] = G[NG - 1 + 8 * p][v];
                            }
                    }
                }
            swept[a] = 1;
        }
        for (int v = 0; v < NV; v++)
            for (int z = 0; z < GS; z++)
                for (int y = 0; y < GS; y++)
                    for (int x = 0; x < GS; x++)
                        L->u_out[cell_index(L, g, v, x, y, z)] =
                            blk[((size_t)(v * PD + z + NG) * PD + y + NG) * PD + x + NG];
        free(blk); free(q); free(o); free(G);
    }
    return err;
}

/* Coarse-fine fix-up of level l (Sec. 2.1, step 3): covered coarse cells
 * become the mean of their 8 children (level l+1 u_out), and leaf coarse
 * cells next to a refined neighbour patch have the coarse face flux replaced
 * by the mean of the 4 fine face fluxes (Berger & Colella).  Corrections of
 * one cell are applied in the order x-, x+, y-, y+, z-, z+. */
int orc_level_fixup(const orc_level *lv, int n_levels, int l, double dt)
{
    if (l < 0 || l + 1 >= n_levels)
        return ORC_ERR_ARG;
    const orc_level *C = &lv[l], *F = &lv[l + 1];
    if (C->child == NULL)
        return ORC_ERR_ARG;
    const double lam = dt / C->dh;
    for (int P = 0; P < 8 * C->n_groups; P++) {
        int g = P / 8, lp = P % 8;
        int pc[3] = {lp & 1, (lp >> 1) & 1, (lp >> 2) & 1};
        int gf = C->child[P];
        if (gf >= 0) {
            /* restriction */
            for (int v = 0; v < NV; v++)
                for (int k = 0; k < PS; k++)
                    for (int j = 0; j < PS; j++)
                        for (int i = 0; i < PS; i++) {
                            double s = 0.0;
                            for (int dz = 0; dz < 2; dz++)
                                for (int dy = 0; dy < 2; dy++)
                                    for (int dx = 0; dx < 2; dx++)
                                        s += F->u_out[cell_index(F, gf, v, 2 * i + dx, 2 * j + dy, 2 * k + dz)];
                            C->u_out[cell_index(C, g, v, PS * pc[0] + i, PS * pc[1] + j, PS * pc[2] + k)] = 0.125 * s;
                        }
            continue;
        }
        if (C->face_flux == NULL || F->face_flux == NULL)
            return ORC_ERR_ARG;
        for (int a = 0; a < 3; a++) {
            int t1 = a == 0 ? 1 : 0, t2 = a == 2 ? 1 : 2;
            for (int s = -1; s <= 1; s += 2) {
                int q[3] = {pc[0], pc[1], pc[2]};
                q[a] += s;
                int gq = g;
                if (q[a] < 0 || q[a] > 1) {
                    int e[3] = {0, 0, 0};
                    e[a] = s;
                    gq = C->nbr[(size_t)g * 26 + dir_index(e[0], e[1], e[2])];
                    q[a] = q[a] < 0 ? 1 : 0;
                }
                if (gq < 0)
                    continue;
                int Q = 8 * gq + (q[2] * 2 + q[1]) * 2 + q[0];
                int gfq = C->child[Q];
                if (gfq < 0)
                    continue;
                int plane_c = s > 0 ? pc[a] + 1 : pc[a];
                int plane_f = s > 0 ? 0 : 2;
                int ca = s > 0 ? PS - 1 : 0;
                for (int v = 0; v < NV; v++)
                    for (int b2 = 0; b2 < PS; b2++)
                        for (int b1 = 0; b1 < PS; b1++) {
                            int T1 = PS * pc[t1] + b1, T2 = PS * pc[t2] + b2;
                            double Gc = C->face_flux[((((size_t)g * 3 + a) * 3 + plane_c) * NV + v) * GS * GS +
                                                     (size_t)T2 * GS + T1];
                            const size_t fo = ((((size_t)gfq * 3 + a) * 3 + plane_f) * NV + v) * GS * GS;
                            const size_t k00 = fo + (size_t)(2 * b2) * GS + 2 * b1, k01 = k00 + 1;
                            const size_t k10 = k00 + GS, k11 = k10 + 1;
                            double f00 = F->face_flux[k00], f01 = F->face_flux[k01];
                            double f10 = F->face_flux[k10], f11 = F->face_flux[k11];
                            if (F->face_flux2 != NULL) {
                                /* individual time steps: mean over the fine level's two steps */
                                f00 = 0.5 * (f00 + F->face_flux2[k00]);
                                f01 = 0.5 * (f01 + F->face_flux2[k01]);
                                f10 = 0.5 * (f10 + F->face_flux2[k10]);
                                f11 = 0.5 * (f11 + F->face_flux2[k11]);
                            }
                            double Gf = 0.25 * (((f00 + f01) + f10) + f11);
                            int xyz[3];
                            xyz[a] = PS * pc[a] + ca;
                            xyz[t1] = T1;
                            xyz[t2] = T2;
                            size_t ci = cell_index(C, g, v, xyz[0], xyz[1], xyz[2]);
                            if (s > 0)
                                C->u_out[ci] = C->u_out[ci] + lam * (Gc - Gf);
                            else
                                C->u_out[ci] = C->u_out[ci] - lam * (Gc - Gf);
                        }
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ regridding */

/* Quantity of the refinement criterion at a group-local position (density
 * or pressure, Eqs. ShockTube_RefineCriterion and BlastWave_RefineCriterion)
 * and a first-order bound on the error of evaluating it in a binary format
 * of unit roundoff u: |fl_u(q) - q| <= u * eq (+ O(u^2)).  With exact inputs
 * the density is exact (eq = 0).  For the pressure of Eqs. ThermalEnergy and
 * EOS, P = (gamma-1)(e - K) with K = rho (vx^2 + vy^2 + vz^2) / 2 and
 * v = m / rho: each velocity carries one rounding, each square three, the
 * sum of three non-negative squares five, the product with rho six, so
 * |fl(K) - K| <= 6 u K; the subtraction adds u |e - K| and the two roundings
 * of gamma - 1 and of the product add 2 u |P| / (gamma - 1).  eq takes
 * (gamma-1)(8 K + 4 |e - K|), above the first-order (gamma-1)(6 K + 3 |e - K|),
 * so that any order of the three-term sum stays inside it.
 * Returns 0 on success, 1 if the position only exists on the coarser level. */
static int crit_value(const orc_level *L, int g, int x, int y, int z, int criterion, double gamma, double *q,
                      double *eq)
{
    double u[NV];
    int r = level_fetch(L, L->u, g, x, y, z, u);
    if (r != 0)
        return r;
    if (criterion != 1) {
        *q = u[0];
        *eq = 0.0;
        return 0;
    }
    *q = orc_pressure(u, gamma);
    const double rho = u[0];
    const double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
    const double K = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    *eq = (gamma - 1.0) * (8.0 * fabs(K) + 4.0 * fabs(u[4] - K));
    return 0;
}

/* The criterion of one cell of level l (group-local position x, y, z of
 * group g; readings R21):
 *   criterion 0 / 1: r = max over the three axes of |q(+1) - q(-1)| / (2 |q|)
 *                    for q = rho / P, a neighbour that only exists on the
 *                    coarser level replaced by the cell itself, NaN ratios
 *                    (0 / 0) skipped, 0 if all are;
 *   criterion 2:     r = rho.
 * *bound gets a first-order bound on the error of the same value evaluated
 * in a format of unit roundoff u_eval, |fl_u(r) - r| <= bound: with
 * n = |q+ - q-| and d = 2 |q0|, fl(n) = (n + dn)(1 + d1), fl(d) = d + dd and
 * a rounded quotient give |fl(r) - r| <= u ((e+ + e-) / d + 2 r e0 / d + 2 r)
 * per axis, and the largest of the per-axis values moves by at most the
 * largest per-axis bound.  The bound is infinite when the denominator itself
 * is not known to one part in four (u 2 e0 > d / 4), where a first-order
 * bound says nothing, and 0 when u_eval is 0. */
static int cell_criterion(const orc_level *L, int g, int x, int y, int z, int criterion, double gamma,
                          double u_eval, double *val, double *bound)
{
    double q0, e0;
    if (crit_value(L, g, x, y, z, criterion == 2 ? 0 : criterion, gamma, &q0, &e0) != 0)
        return ORC_ERR_MAP;
    if (criterion == 2) {
        *val = q0;
        *bound = 0.0;
        return ORC_OK;
    }
    const int c[3] = {x, y, z};
    const double d = 2.0 * fabs(q0);
    double rmax = 0.0, emax = 0.0;
    for (int a = 0; a < 3; a++) {
        double qm, qp, em, ep;
        int m[3] = {c[0], c[1], c[2]}, pp[3] = {c[0], c[1], c[2]};
        m[a] -= 1;
        pp[a] += 1;
        int rm = crit_value(L, g, m[0], m[1], m[2], criterion, gamma, &qm, &em);
        int rp = crit_value(L, g, pp[0], pp[1], pp[2], criterion, gamma, &qp, &ep);
        if (rm < 0 || rp < 0)
            return ORC_ERR_MAP;
        if (rm == 1) {
            qm = q0;
            em = e0;
        }
        if (rp == 1) {
            qp = q0;
            ep = e0;
        }
        double r = fabs(qp - qm) / d;
        if (r > rmax)
            rmax = r;
        double ea = (ep + em) / d;
        if (ea > emax)
            emax = ea;
    }
    /* the r terms with the largest r bound those of every axis */
    double b = u_eval * (emax + 2.0 * rmax * e0 / d + 2.0 * rmax);
    if (u_eval > 0.0 && !(u_eval * 2.0 * e0 <= 0.25 * d))
        b = INFINITY;
    *val = rmax;
    *bound = b;
    return ORC_OK;
}

/* Per cell of level l the criterion value and the bound on its error at
 * unit roundoff u_eval (cell_criterion), in the level's storage order
 * [8 n_groups][8][8][8]. */
int orc_flag_criterion(const orc_level *lv, int n_levels, int l, double gamma, int criterion, double u_eval,
                       double *val, double *bound)
{
    if (l < 0 || l >= n_levels || criterion < 0 || criterion > 2)
        return ORC_ERR_ARG;
    const orc_level *L = &lv[l];
    for (int g = 0; g < L->n_groups; g++)
        for (int z = 0; z < GS; z++)
            for (int y = 0; y < GS; y++)
                for (int x = 0; x < GS; x++) {
                    size_t k = cell_index(L, g, 0, x, y, z);
                    int r = cell_criterion(L, g, x, y, z, criterion, gamma, u_eval, &val[k], &bound[k]);
                    if (r != ORC_OK)
                        return r;
                }
    return ORC_OK;
}

/* Flag buffer of one flagged cell (reading R22): the bit of every patch
 * offset (dx,dy,dz) that the cube of 1 + 2 n_buffer cells around the cell
 * reaches, bit (dz+1)*9 + (dy+1)*3 + (dx+1), into the mask of its patch. */
static void buffer_bits(int g, int x, int y, int z, int n_buffer, uint32_t *masks)
{
    int lp = ((z / PS) * 2 + (y / PS)) * 2 + (x / PS);
    int pc[3] = {x % PS, y % PS, z % PS};
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = pc[a] - n_buffer < 0 ? -1 : 0;
        hi[a] = pc[a] + n_buffer > PS - 1 ? 1 : 0;
    }
    uint32_t m = 0u;
    for (int dz = lo[2]; dz <= hi[2]; dz++)
        for (int dy = lo[1]; dy <= hi[1]; dy++)
            for (int dx = lo[0]; dx <= hi[0]; dx++)
                m |= 1u << ((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
    masks[8 * g + lp] |= m;
}

/* Flag step of the refinement-map rebuild (Sec. 2.1 step 4; readings R21,
 * R22).  A cell of level l is flagged when its criterion value r
 * (cell_criterion) reaches the threshold: r >= threshold for the gradient
 * criteria 0 (density) and 1 (pressure), r > threshold for criterion 2
 * (density).  Around every such cell the flag buffer (buffer_bits) marks
 * the patches it reaches; masks[p] of patch p gets their bits (bit 13: p
 * itself).  0 <= n_buffer <= 8.  The decision is taken in double precision
 * on the level's values.
 *
 * u_eval > 0 asks, in addition, for the decisions that an evaluation of
 * the criterion in a format of unit roundoff u_eval could take: a cell
 * whose value lies within the error bound of cell_criterion of the
 * threshold may go either way.  masks gets the flags of the cells flagged whatever the
 * rounding, masks_maybe (may be NULL when u_eval == 0) those of the cells
 * that may be flagged, and *n_near (may be NULL) the number of cells that
 * may go either way.  u_eval == 0: the plain double decision in both. */
int orc_flag_level(const orc_level *lv, int n_levels, int l, double gamma, int criterion, double threshold,
                   int n_buffer, double u_eval, uint32_t *masks, uint32_t *masks_maybe, int64_t *n_near)
{
    if (l < 0 || l >= n_levels || n_buffer < 0 || n_buffer > PS || criterion < 0 || criterion > 2 ||
        !(u_eval >= 0.0))
        return ORC_ERR_ARG;
    const orc_level *L = &lv[l];
    for (int p = 0; p < 8 * L->n_groups; p++) {
        masks[p] = 0u;
        if (masks_maybe != NULL)
            masks_maybe[p] = 0u;
    }
    int64_t near = 0;
    for (int g = 0; g < L->n_groups; g++)
        for (int z = 0; z < GS; z++)
            for (int y = 0; y < GS; y++)
                for (int x = 0; x < GS; x++) {
                    double r, b;
                    int rc = cell_criterion(L, g, x, y, z, criterion, gamma, u_eval, &r, &b);
                    if (rc != ORC_OK)
                        return rc;
                    int hit = criterion == 2 ? r > threshold : r >= threshold;
                    int sure = hit, maybe = hit;
                    if (u_eval > 0.0) {
                        if (criterion == 2) {
                            sure = r - b > threshold;
                            maybe = r + b > threshold;
                        } else {
                            sure = r - b >= threshold;
                            maybe = r + b >= threshold;
                        }
                    }
                    if (sure != maybe)
                        near++;
                    if (sure)
                        buffer_bits(g, x, y, z, n_buffer, masks);
                    if (maybe && masks_maybe != NULL)
                        buffer_bits(g, x, y, z, n_buffer, masks_maybe);
                }
    if (n_near != NULL)
        *n_near = near;
    return ORC_OK;
}

/* Refinement step (Sec. 2.1 step 4): the data of a rebuilt level.  lv[0..l]
 * are the levels up to the new level's parent level l; the new level has
 * n_new groups whose parents (patches of level l) are parent_new.  Group i
 * copies old group inherit[i] of the previous fine level (u_old, n_old
 * groups) when inherit[i] >= 0, and otherwise fills every cell by Min-Mod
 * interpolation from level l (R8), into u_new. */
int orc_refine_fill(const orc_level *lv, int l, int n_new, const int32_t *parent_new,
                    const int32_t *inherit, const double *u_old, int n_old, double *u_new)
{
    orc_level tmp[MAXLV + 1];
    if (l < 0 || l >= MAXLV)
        return ORC_ERR_ARG;
    for (int k = 0; k <= l; k++) {
        tmp[k] = lv[k];
        tmp[k].u_new = NULL;
        tmp[k].coarse_w = 0.0;
    }
    orc_level *F = &tmp[l + 1];
    memset(F, 0, sizeof(*F));
    F->n_groups = n_new;
    F->dh = 0.5 * lv[l].dh;
    F->parent = parent_new;
    F->u_out = u_new;
    const size_t cells = (size_t)PS * PS * PS;
    for (int i = 0; i < n_new; i++) {
        if (inherit[i] >= 0) {
            if (inherit[i] >= n_old)
                return ORC_ERR_ARG;
            for (int v = 0; v < NV; v++)
                memcpy(u_new + ((size_t)v * 8 * n_new + 8 * (size_t)i) * cells,
                       u_old + ((size_t)v * 8 * n_old + 8 * (size_t)inherit[i]) * cells,
                       sizeof(double) * 8 * cells);
            continue;
        }
        for (int z = 0; z < GS; z++)
            for (int y = 0; y < GS; y++)
                for (int x = 0; x < GS; x++) {
                    double val[NV];
                    if (prolong_fetch(tmp, l + 1, i, x, y, z, val) != 0)
                        return ORC_ERR_MAP;
                    for (int v = 0; v < NV; v++)
                        u_new[cell_index(F, i, v, x, y, z)] = val[v];
                }
    }
    return ORC_OK;
}

/* ----------------------------------------------------- Poisson (SOR) */

/* Red-black successive overrelaxation for one patch group (Sec. 2.3, Eqs.
 * Residual and SOR; reading R24).  phi: [18][18][18] (x fastest) holding
 * the Dirichlet ghost layer, which is kept, and the initial interior; rho:
 * [16][16][16]; coef = 4 pi G dh^2.  One iteration updates the even
 * interior cells (i + j + k even, interior indices 0..15) with
 *   R = (phi(i+1) + phi(j+1) + phi(k+1) + phi(i-1) + phi(j-1) + phi(k-1)
 *        - 6 phi) - coef rho,   phi <- phi + (omega / 6) R,
 * and then the odd cells with the updated even values.  It stops after the
 * iteration in which the one-norm of that iteration's residuals falls to
 * tol times the one-norm of coef rho, or after max_iter iterations (tol = 0
 * asks for exactly max_iter iterations), and returns the number of
 * iterations; *res gets the last residual norm. */
int orc_sor_group(double *phi, const double *rho, double coef, double omega, int max_iter, double tol,
                  double *res)
{
    const int P = GS + 2;
    double src = 0.0;
    for (int i = 0; i < GS * GS * GS; i++)
        src += fabs(coef * rho[i]);
    const double w6 = omega / 6.0;
    double norm = 0.0;
    int it = 0;
    while (it < max_iter) {
        norm = 0.0;
        for (int color = 0; color < 2; color++)
            for (int k = 0; k < GS; k++)
                for (int j = 0; j < GS; j++)
                    for (int i = 0; i < GS; i++) {
                        if (((i + j + k) & 1) != color)
                            continue;
                        const int c = ((k + 1) * P + (j + 1)) * P + (i + 1);
                        const double nb = ((((phi[c + 1] + phi[c + P]) + phi[c + P * P]) + phi[c - 1]) + phi[c - P]) +
                                          phi[c - P * P];
                        const double R = (nb - 6.0 * phi[c]) - coef * rho[(k * GS + j) * GS + i];
                        phi[c] = phi[c] + w6 * R;
                        norm += fabs(R);
                    }
        it++;
        if (tol > 0.0 && norm <= tol * src)
            break;
    }
    *res = norm;
    return it;
}

/* Inputs of the SOR solver of level l >= 1 (Sec. 2.3; reading R26): for
 * every patch group g of level l, phi_blk[g] ([18][18][18], x fastest) is
 * the Min-Mod interpolation (reading R8) of the coarser level's potential
 * phi_c ([8 n_c][8][8][8], the level layout) at every cell of the group and
 * of its one-cell ghost layer -- the ghost layer is the Dirichlet boundary of
 * the group's problem, which the paper fills from the level one coarser,
 * the interior the initial guess -- and rho_blk[g] ([16][16][16], x fastest)
 * is the group's density from the level's state. */
int orc_poisson_prepare(const orc_level *lv, int n_levels, int l, const double *phi_c, double *phi_blk,
                        double *rho_blk)
{
    if (l < 1 || l >= n_levels || n_levels > MAXLV)
        return ORC_ERR_ARG;
    const int P = GS + 2;
    orc_level tmp[MAXLV];
    memcpy(tmp, lv, (size_t)n_levels * sizeof(orc_level));
    /* the coarser level with the potential as its variable 0 (the other
     * variables are interpolated alongside and dropped) */
    const size_t ncell_c = (size_t)lv[l - 1].n_groups * 8 * PS * PS * PS;
    double *uc = (double *)calloc(NV * ncell_c, sizeof(double));
    if (uc == NULL)
        return ORC_ERR_ARG;
    memcpy(uc, phi_c, ncell_c * sizeof(double));
    tmp[l - 1].u = uc;
    tmp[l - 1].u_new = NULL;
    tmp[l].coarse_w = 0.0;
    int err = 0;
    for (int g = 0; g < lv[l].n_groups && !err; g++) {
        for (int z = -1; z <= GS && !err; z++)
            for (int y = -1; y <= GS && !err; y++)
                for (int x = -1; x <= GS; x++) {
                    double val[NV];
                    if (prolong_fetch(tmp, l, g, x, y, z, val) != 0) {
                        err = 1;
                        break;
                    }
                    phi_blk[(size_t)g * P * P * P + ((z + 1) * P + (y + 1)) * P + (x + 1)] = val[0];
                }
        for (int z = 0; z < GS; z++)
            for (int y = 0; y < GS; y++)
                for (int x = 0; x < GS; x++)
                    rho_blk[(size_t)g * GS * GS * GS + (z * GS + y) * GS + x] = lv[l].u[cell_index(&lv[l], g, 0, x, y, z)];
    }
    free(uc);
    return err ? ORC_ERR_MAP : ORC_OK;
}

/* ------------------------------------------------------- gravity (G) */

/* The gravity operator G of the split scheme (Sec. 2.3: Eqs. MomConserve
 * and EnergyConserve with their flux terms dropped; reading R25), over dt,
 * on one level.  u: [5][8 n_groups][8][8][8], updated in place; phi:
 * [n_groups][18][18][18] (x fastest), the potential of each patch group
 * with one layer of ghost cells.  Per cell, along each axis k the 3-point
 * central difference gives d_k = (phi(-1) - phi(+1)) lam = g_k dt with
 * lam = dt / (2 dh); then
 *   m_k <- m_k + rho d_k                                   (k = x, y, z)
 *   e   <- e + 0.5 (((m_x + m'_x) d_x + (m_y + m'_y) d_y) + (m_z + m'_z) d_z)
 * with m' the new momentum.  Over the step rho and g are constant, so this
 * is the exact solution of the split equations; it changes the kinetic
 * energy only, never the thermal energy. */
void orc_gravity_level(double *u, int n_groups, const double *phi, double dh, double dt)
{
    const int P = GS + 2;
    const double lam = dt / (2.0 * dh);
    orc_level L;
    memset(&L, 0, sizeof(L));
    L.n_groups = n_groups;
#pragma omp parallel for schedule(static)
    for (int g = 0; g < n_groups; g++) {
        const double *ph = phi + (size_t)g * P * P * P;
        for (int z = 0; z < GS; z++)
            for (int y = 0; y < GS; y++)
                for (int x = 0; x < GS; x++) {
                    const int c = ((z + 1) * P + (y + 1)) * P + (x + 1);
                    const int st[3] = {1, P, P * P};
                    size_t off[NV];
                    for (int v = 0; v < NV; v++)
                        off[v] = cell_index(&L, g, v, x, y, z);
                    const double rho = u[off[0]];
                    double d[3], m0[3], m1[3];
                    for (int k = 0; k < 3; k++) {
                        d[k] = (ph[c - st[k]] - ph[c + st[k]]) * lam;
                        m0[k] = u[off[1 + k]];
                        m1[k] = m0[k] + rho * d[k];
                    }
                    const double de = ((m0[0] + m1[0]) * d[0] + (m0[1] + m1[1]) * d[1]) + (m0[2] + m1[2]) * d[2];
                    for (int k = 0; k < 3; k++)
                        u[off[1 + k]] = m1[k];
                    u[off[4]] = u[off[4]] + 0.5 * de;
                }
    }
}

/* ------------------------------------------------------ CFL and checks */

/* Largest signal speed c_s + max(|vx|,|vy|,|vz|) over all cells of level l
 * (denominator of Eq. CFL). */
double orc_level_max_speed(const orc_level *L, double gamma)
{
    double smax = 0.0;
    size_t ncell = (size_t)L->n_groups * 8 * PS * PS * PS;
    for (size_t i = 0; i < ncell; i++) {
        double u[NV];
        for (int v = 0; v < NV; v++)
            u[v] = L->u[v * ncell + i];
        double rho = u[0];
        double vx = u[1] / rho, vy = u[2] / rho, vz = u[3] / rho;
        double eps = u[4] - 0.5 * rho * (vx * vx + vy * vy + vz * vz);
        double P = (gamma - 1.0) * eps;
        double cs = sqrt(gamma * fmax(P, 0.0) / rho);
        double s = cs + fmax(fmax(fabs(vx), fabs(vy)), fabs(vz));
        if (s > smax || s != s)
            smax = s;
        if (smax != smax)
            break;
    }
    return smax;
}

/* Eq. CFL with a safety factor: dt = cfl * min over levels of dh_l / s_l. */
double orc_cfl_dt_steps(const orc_level *lv, int n_levels, double gamma, double cfl, int individual);

double orc_cfl_dt(const orc_level *lv, int n_levels, double gamma, double cfl)
{
    return orc_cfl_dt_steps(lv, n_levels, gamma, cfl, 0);
}

/* Eq. CFL for the step of level 0: with individual time steps (individual
 * != 0) level l takes 2^l steps per level-0 step, so its condition
 * dt / 2^l <= cfl dh_l / s_l bounds the level-0 dt by cfl 2^l dh_l / s_l. */
double orc_cfl_dt_steps(const orc_level *lv, int n_levels, double gamma, double cfl, int individual)
{
    double dt = INFINITY;
    for (int l = 0; l < n_levels; l++) {
        if (lv[l].n_groups == 0)
            continue;
        double s = orc_level_max_speed(&lv[l], gamma);
        double d = (individual ? ldexp(lv[l].dh, l) : lv[l].dh) / s;
        if (d < dt || d != d)
            dt = d;
    }
    return cfl * dt;
}

/* Sums of u * dV over leaf cells of all levels and the number of leaf cells
 * with rho <= 0, P <= 0 or a non-finite conserved variable. */
int orc_check(const orc_level *lv, int n_levels, double gamma, double *sums,
              int64_t *n_bad)
{
    for (int v = 0; v < NV; v++)
        sums[v] = 0.0;
    *n_bad = 0;
    for (int l = 0; l < n_levels; l++) {
        const orc_level *L = &lv[l];
        size_t ncell = (size_t)L->n_groups * 8 * PS * PS * PS;
        double dV = L->dh * L->dh * L->dh;
        for (size_t i = 0; i < ncell; i++) {
            size_t patch = i / (PS * PS * PS);
            if (L->child && L->child[patch] >= 0)
                continue;
            double u[NV];
            int finite = 1;
            for (int v = 0; v < NV; v++) {
                u[v] = L->u[v * ncell + i];
                sums[v] += u[v] * dV;
                finite &= isfinite(u[v]) ? 1 : 0;
            }
            if (!finite || !(u[0] > 0.0) || !(orc_pressure(u, gamma) > 0.0))
                (*n_bad)++;
        }
    }
    return ORC_OK;
}

/* Exported for the ghost-zone tests: the padded 22^3 block of group g of
 * level l, blk[NV][22][22][22] (x fastest). */
int orc_gather_block(const orc_level *lv, int n_levels, int l, int g, double *blk)
{
    if (l < 0 || l >= n_levels || g < 0 || g >= lv[l].n_groups)
        return ORC_ERR_ARG;
    return gather_block(lv, l, g, blk);
}
