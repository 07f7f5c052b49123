/*
 * pic_oracle.c -- plain, slow FP64 CPU oracle of the implicit 2D3V PIC step of
 * Petrov & Davis, "Parallelization of an implicit algorithm for
 * multi-dimensional particle-in-cell simulations" (Section 2, Eqs. 1-5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code; the CUDA library never
 * does, and this file shares no code with it.
 *
 * Every routine is a direct loop over particles, nodes or cells, in the order
 * the equations are written, with no blocking or fusion.
 *
 * Units: c = eps0 = mu0 = 1 (so B = H), u = p/(m c), time in 1/omega_r.
 *
 * Grid (Section 3.2, Fig. 1): nx x ny cells of size dx x dy.  E and the
 * deposited moments live on nodes (i*dx, j*dy); H lives at cell centres
 * ((i+1/2)dx, (j+1/2)dy).  y is always periodic.  Along x the box is either
 * periodic (nxn = nx node columns) or bounded by absorbing walls
 * (nxn = nx + 1 node columns, columns 0 and nx on the walls).
 * Arrays are planar: component c of node (i, j) is at [c*ny*nxn + j*nxn + i];
 * component c of cell (i, j) at [c*ny*nx + j*nx + i].
 *
 * Moment planes (13 per node): 0 = rho; 1..9 = S_xx S_xy S_xz S_yx S_yy S_yz
 * S_zx S_zy S_zz (row = component of j, column = component of E);
 * 10..12 = dj_x dj_y dj_z.
 *
 * Shape function W (the paper's Section 3.3, last paragraph): order 1 is the
 * paper's linear area weighting over the particle's cell; orders 2, 3 and 4,
 * the higher-order polynomial shapes the paper mentions (up to fourth order),
 * are the centred B-splines of that degree over the (n + 1) x (n + 1) nodes
 * nearest the particle.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NMOM 13

static int node_cols(int nx, int periodic_x) { return periodic_x ? nx : nx + 1; }

/* Cell index and in-cell fraction of coordinate s (in cell units) on an axis
 * of n cells.  floor/fraction as written; a coordinate that rounds onto the
 * far edge is folded back (periodic) or, inside a wall (x < Lx whose x/dx
 * rounds to n), put in the last cell at the largest fraction below 1, so that
 * every fraction lies in [0, 1). */
static void locate(double s, int n, int periodic, int *c, double *f)
{
    double fl = floor(s);
    int ci = (int)fl;
    double fr = s - fl;
    if (ci >= n) {
        if (periodic) { ci -= n; } else { ci = n - 1; fr = nextafter(1.0, 0.0); }
    }
    if (ci < 0) {
        if (periodic) { ci += n; } else { ci = 0; fr = 0.0; }
    }
    *c = ci;
    *f = fr;
}

/* The four corner nodes of a particle's cell and their area weights
 * (linear weighting within the cell, Section 3.3 last paragraph). */
static void corners(int nx, int ny, int periodic_x, double dx, double dy, double x, double y,
                    int64_t node[4], double W[4])
{
    int nxn = node_cols(nx, periodic_x);
    int ci, cj;
    double fx, fy;
    locate(x / dx, nx, periodic_x, &ci, &fx);
    locate(y / dy, ny, 1, &cj, &fy);
    int i0 = ci, i1 = ci + 1;
    if (periodic_x && i1 == nx) i1 = 0;
    int j0 = cj, j1 = (cj + 1 == ny) ? 0 : cj + 1;
    node[0] = (int64_t)j0 * nxn + i0; W[0] = (1.0 - fx) * (1.0 - fy);
    node[1] = (int64_t)j0 * nxn + i1; W[1] = fx * (1.0 - fy);
    node[2] = (int64_t)j1 * nxn + i0; W[2] = (1.0 - fx) * fy;
    node[3] = (int64_t)j1 * nxn + i1; W[3] = fx * fy;
}

/* Centred B-spline of degree n (2, 3 or 4) at x (in cells), from its
 * piecewise polynomial form. */
static double bspline(int n, double x)
{
    double a = fabs(x);
    if (n == 2) {
        if (a <= 0.5) return 0.75 - a * a;
        if (a <= 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
        return 0.0;
    }
    if (n == 3) {
        if (a <= 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
        if (a <= 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
        return 0.0;
    }
    if (a <= 0.5) return 115.0 / 192.0 - 0.625 * a * a + 0.25 * a * a * a * a;
    if (a <= 1.5) return (55.0 + 20.0 * a - 120.0 * a * a + 80.0 * a * a * a - 16.0 * a * a * a * a) / 96.0;
    if (a <= 2.5) { double b = 5.0 - 2.0 * a; return b * b * b * b / 384.0; }
    return 0.0;
}

/* B-spline weights of degree n along one axis for a particle in cell c at
 * fraction f: the n + 1 nodes from the first one within (n + 1)/2 of the
 * particle (odd n: c - (n - 1)/2; even n: c - n/2, or one more when f >= 1/2,
 * i.e. centred on the nearest node), each weighted by the spline at its
 * distance (node - c) - f.  Node indices are returned unwrapped. */
static void spline_axis(int n, int c, double f, int idx[5], double w[5])
{
    int first = (n % 2) ? c - (n - 1) / 2 : c - n / 2 + (f >= 0.5 ? 1 : 0);
    for (int k = 0; k <= n; ++k) {
        idx[k] = first + k;
        w[k] = bspline(n, (double)(first + k - c) - f);
    }
}

/* Node index along an axis of n cells: periodic wrap, or (x with walls) a node
 * beyond a wall folded onto the wall node (reading: its weight stays in the box). */
static int axis_node(int i, int n, int periodic)
{
    if (periodic) return ((i % n) + n) % n;
    if (i < 0) return 0;
    if (i > n) return n;
    return i;
}

#define MAX_SHAPE_NODES 25

/* The nodes of a particle and their weights for shape order 1 (the cell's 4
 * corners) or n = 2..4 ((n + 1) x (n + 1) spline nodes; a node folded onto a
 * wall appears more than once).  Returns the number of entries. */
static int shape_nodes(int order, int nx, int ny, int periodic_x, double dx, double dy, double x, double y,
                       int64_t node[MAX_SHAPE_NODES], double W[MAX_SHAPE_NODES])
{
    if (order < 2) {
        corners(nx, ny, periodic_x, dx, dy, x, y, node, W);
        return 4;
    }
    int nxn = node_cols(nx, periodic_x);
    int ci, cj;
    double fx, fy;
    locate(x / dx, nx, periodic_x, &ci, &fx);
    locate(y / dy, ny, 1, &cj, &fy);
    int ix[5], iy[5];
    double wx[5], wy[5];
    spline_axis(order, ci, fx, ix, wx);
    spline_axis(order, cj, fy, iy, wy);
    int k = 0;
    for (int b = 0; b <= order; ++b)
        for (int a = 0; a <= order; ++a) {
            node[k] = (int64_t)axis_node(iy[b], ny, 1) * nxn + axis_node(ix[a], nx, periodic_x);
            W[k] = wx[a] * wy[b];
            ++k;
        }
    return k;
}

/* Node indices and weights of a batch of positions (for the shape pins):
 * MAX_SHAPE_NODES entries per particle, unused ones -1 and 0. */
void orc_shape_nodes(int nx, int ny, int periodic_x, double dx, double dy, int order, int64_t np,
                     const double *x, const double *y, int64_t *node, double *W)
{
    for (int64_t p = 0; p < np; ++p) {
        int64_t nd[MAX_SHAPE_NODES];
        double w[MAX_SHAPE_NODES];
        int n = shape_nodes(order, nx, ny, periodic_x, dx, dy, x[p], y[p], nd, w);
        for (int k = 0; k < MAX_SHAPE_NODES; ++k) {
            node[MAX_SHAPE_NODES * p + k] = k < n ? nd[k] : -1;
            W[MAX_SHAPE_NODES * p + k] = k < n ? w[k] : 0.0;
        }
    }
}

/* Cell and in-cell fraction of a batch of positions (for ordering and tests). */
void orc_locate(int nx, int ny, int periodic_x, double dx, double dy, int64_t np,
                const double *x, const double *y, int32_t *cx, int32_t *cy, double *fx, double *fy)
{
    for (int64_t p = 0; p < np; ++p) {
        int a, b;
        double f, g;
        locate(x[p] / dx, nx, periodic_x, &a, &f);
        locate(y[p] / dy, ny, 1, &b, &g);
        cx[p] = a; cy[p] = b; fx[p] = f; fy[p] = g;
    }
}

/* Gather (a2): value of a 3-component node field at each particle. */
void orc_gather(int nx, int ny, int periodic_x, double dx, double dy, const double *F,
                int64_t np, const double *x, const double *y, double *out, int order)
{
    int64_t plane = (int64_t)ny * node_cols(nx, periodic_x);
    for (int64_t p = 0; p < np; ++p) {
        int64_t nd[MAX_SHAPE_NODES];
        double W[MAX_SHAPE_NODES];
        int n = shape_nodes(order, nx, ny, periodic_x, dx, dy, x[p], y[p], nd, W);
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += W[k] * F[c * plane + nd[k]];
            out[3 * p + c] = s;
        }
    }
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* R(b) v = (v + v x b + (v.b) b) / (1 + |b|^2): the solution ubar of
 * ubar = v + ubar x b, i.e. Eq. 2a written time-centred with the magnetic
 * term evaluated at the mean momentum. */
static void rotate(const double b[3], const double v[3], double o[3])
{
    double vxb[3];
    cross3(v, b, vxb);
    double vb = dot3(v, b);
    double den = 1.0 + dot3(b, b);
    for (int c = 0; c < 3; ++c) o[c] = (v[c] + vxb[c] + vb * b[c]) / den;
}

/* Exported for the pin tests: R(b) applied to v. */
void orc_rotate(const double *b, const double *v, double *o) { rotate(b, v, o); }

/*
 * Implicit push (a3), Eq. 2a-c with the electric field factored out
 * (Section 2): with gamma^n = sqrt(1 + |u^n|^2), k = q dt / (2 m),
 * b = k B / gamma^n and w = u^n + k E^{n+1/2},
 *     ubar = R(b) w,  u^{n+1} = 2 ubar - u^n,  r^{n+1} = r^n + dt ubar / gamma^n
 * (x and y only; nothing depends on z).  E and B are gathered at r^n.  y wraps;
 * x wraps in a periodic box, and a particle leaving [0, Lx) of a walled box is
 * marked dead (alive[p] = 0).
 */
void orc_push(int nx, int ny, int periodic_x, double dx, double dy, double dt, double q, double m,
              const double *Ehalf, const double *Bold, int64_t np,
              double *x, double *y, double *ux, double *uy, double *uz, uint8_t *alive, int order)
{
    int64_t plane = (int64_t)ny * node_cols(nx, periodic_x);
    double Lx = nx * dx, Ly = ny * dy;
    double k = q * dt / (2.0 * m);
    for (int64_t p = 0; p < np; ++p) {
        int64_t nd[MAX_SHAPE_NODES];
        double W[MAX_SHAPE_NODES];
        int n = shape_nodes(order, nx, ny, periodic_x, dx, dy, x[p], y[p], nd, W);
        double E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < n; ++j) {
                E[c] += W[j] * Ehalf[c * plane + nd[j]];
                B[c] += W[j] * Bold[c * plane + nd[j]];
            }
        double u[3] = {ux[p], uy[p], uz[p]};
        double g = sqrt(1.0 + dot3(u, u));
        double b[3], w[3], ub[3];
        for (int c = 0; c < 3; ++c) {
            b[c] = k * B[c] / g;
            w[c] = u[c] + k * E[c];
        }
        rotate(b, w, ub);
        ux[p] = 2.0 * ub[0] - u[0];
        uy[p] = 2.0 * ub[1] - u[1];
        uz[p] = 2.0 * ub[2] - u[2];
        double xn = x[p] + dt * ub[0] / g;
        double yn = y[p] + dt * ub[1] / g;
        yn -= Ly * floor(yn / Ly);
        if (periodic_x) {
            xn -= Lx * floor(xn / Lx);
        } else if (xn < 0.0 || xn >= Lx) {
            if (alive) alive[p] = 0;
        }
        x[p] = xn;
        y[p] = yn;
    }
}

/*
 * Deposit of the implicit source moments (a4), Eq. 3: the current of
 * particle alpha at its next push is j = n q ubar / gamma = S_alpha E + dj_alpha
 * with ubar = R (u + k E), so per particle
 *     rho += W w q,
 *     S   += W w q^2 dt^2 / (4 m gamma) R(b)     (9 components),
 *     dj  += W w q R(b) u / gamma                  (3 components),
 * with gamma = sqrt(1 + |u|^2) and b = q dt B / (2 m gamma), B gathered at the
 * particle.  S here already carries the dt/2 of Eq. 4 (S = dt sigma / 2).
 * Sums are raw (not divided by the node area) and are ADDED to M.
 */
void orc_deposit(int nx, int ny, int periodic_x, double dx, double dy, double dt, double q, double m,
                 const double *Bn, int64_t np, const double *x, const double *y,
                 const double *ux, const double *uy, const double *uz, const double *w,
                 double *M, int order)
{
    int64_t plane = (int64_t)ny * node_cols(nx, periodic_x);
    for (int64_t p = 0; p < np; ++p) {
        int64_t nd[MAX_SHAPE_NODES];
        double W[MAX_SHAPE_NODES];
        int n = shape_nodes(order, nx, ny, periodic_x, dx, dy, x[p], y[p], nd, W);
        double B[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < n; ++j) B[c] += W[j] * Bn[c * plane + nd[j]];
        double u[3] = {ux[p], uy[p], uz[p]};
        double g = sqrt(1.0 + dot3(u, u));
        double b[3];
        for (int c = 0; c < 3; ++c) b[c] = q * dt * B[c] / (2.0 * m * g);
        /* columns of R(b) */
        double R[3][3];
        for (int col = 0; col < 3; ++col) {
            double e[3] = {0, 0, 0}, r[3];
            e[col] = 1.0;
            rotate(b, e, r);
            for (int row = 0; row < 3; ++row) R[row][col] = r[row];
        }
        double Ru[3];
        rotate(b, u, Ru);
        double vals[NMOM];
        vals[0] = w[p] * q;
        double cs = w[p] * q * q * dt * dt / (4.0 * m * g);
        for (int row = 0; row < 3; ++row)
            for (int col = 0; col < 3; ++col) vals[1 + 3 * row + col] = cs * R[row][col];
        for (int c = 0; c < 3; ++c) vals[10 + c] = w[p] * q * Ru[c] / g;
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < NMOM; ++k) M[k * plane + nd[j]] += W[j] * vals[k];
    }
}

/* Area attached to node column i: dx dy, halved on a wall column. */
static double node_area(int nx, int periodic_x, double dx, double dy, int i)
{
    if (!periodic_x && (i == 0 || i == nx)) return 0.5 * dx * dy;
    return dx * dy;
}

/* Divide raw node sums by the node area (reading of "accumulated on grid nodes"). */
void orc_normalize(int nx, int ny, int periodic_x, double dx, double dy, const double *Mraw, double *Mout)
{
    int nxn = node_cols(nx, periodic_x);
    int64_t plane = (int64_t)ny * nxn;
    for (int k = 0; k < NMOM; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nxn; ++i) {
                int64_t id = k * plane + (int64_t)j * nxn + i;
                Mout[id] = Mraw[id] / node_area(nx, periodic_x, dx, dy, i);
            }
}

/*
 * curl of the cell-centred H at the nodes: centred differences over the four
 * cells that share the node, e.g. dHz/dy at node (i,j) =
 * [(Hz(i,j) + Hz(i-1,j)) - (Hz(i,j-1) + Hz(i-1,j-1))] / (2 dy), cell (i,j) being
 * the one whose lower-left corner is node (i,j); d/dz = 0.  On a wall column
 * only the two cells inside the box exist: there dHz/dy and dHx/dy are formed
 * from them and the x-derivatives are left out (those terms are set to 0).
 */
void orc_curl_h(int nx, int ny, int periodic_x, double dx, double dy, const double *H, double *out)
{
    int nxn = node_cols(nx, periodic_x);
    int64_t cp = (int64_t)ny * nx, np_ = (int64_t)ny * nxn;
    for (int j = 0; j < ny; ++j) {
        int jm = (j == 0) ? ny - 1 : j - 1;
        for (int i = 0; i < nxn; ++i) {
            int64_t o = (int64_t)j * nxn + i;
            if (!periodic_x && (i == 0 || i == nx)) {
                int ic = (i == 0) ? 0 : nx - 1;
                double hz_up = H[2 * cp + (int64_t)j * nx + ic], hz_dn = H[2 * cp + (int64_t)jm * nx + ic];
                double hx_up = H[0 * cp + (int64_t)j * nx + ic], hx_dn = H[0 * cp + (int64_t)jm * nx + ic];
                out[0 * np_ + o] = (hz_up - hz_dn) / dy;
                out[1 * np_ + o] = 0.0;
                out[2 * np_ + o] = -(hx_up - hx_dn) / dy;
                continue;
            }
            int im = (i == 0) ? nx - 1 : i - 1;
            int64_t a = (int64_t)j * nx + i;    /* upper right */
            int64_t b = (int64_t)j * nx + im;   /* upper left  */
            int64_t c = (int64_t)jm * nx + i;   /* lower right */
            int64_t d = (int64_t)jm * nx + im;  /* lower left  */
            double dHz_dy = ((H[2 * cp + a] + H[2 * cp + b]) - (H[2 * cp + c] + H[2 * cp + d])) / (2.0 * dy);
            double dHz_dx = ((H[2 * cp + a] + H[2 * cp + c]) - (H[2 * cp + b] + H[2 * cp + d])) / (2.0 * dx);
            double dHy_dx = ((H[1 * cp + a] + H[1 * cp + c]) - (H[1 * cp + b] + H[1 * cp + d])) / (2.0 * dx);
            double dHx_dy = ((H[0 * cp + a] + H[0 * cp + b]) - (H[0 * cp + c] + H[0 * cp + d])) / (2.0 * dy);
            out[0 * np_ + o] = dHz_dy;
            out[1 * np_ + o] = -dHz_dx;
            out[2 * np_ + o] = dHy_dx - dHx_dy;
        }
    }
}

/* curl of the nodal E at the cell centres, from the cell's four corner nodes. */
void orc_curl_e(int nx, int ny, int periodic_x, double dx, double dy, const double *E, double *out)
{
    int nxn = node_cols(nx, periodic_x);
    int64_t cp = (int64_t)ny * nx, np_ = (int64_t)ny * nxn;
    for (int j = 0; j < ny; ++j) {
        int jp = (j + 1 == ny) ? 0 : j + 1;
        for (int i = 0; i < nx; ++i) {
            int ip = i + 1;
            if (periodic_x && ip == nx) ip = 0;
            int64_t p00 = (int64_t)j * nxn + i, p10 = (int64_t)j * nxn + ip;
            int64_t p01 = (int64_t)jp * nxn + i, p11 = (int64_t)jp * nxn + ip;
            double dEz_dy = ((E[2 * np_ + p01] + E[2 * np_ + p11]) - (E[2 * np_ + p00] + E[2 * np_ + p10])) / (2.0 * dy);
            double dEz_dx = ((E[2 * np_ + p10] + E[2 * np_ + p11]) - (E[2 * np_ + p00] + E[2 * np_ + p01])) / (2.0 * dx);
            double dEy_dx = ((E[1 * np_ + p10] + E[1 * np_ + p11]) - (E[1 * np_ + p00] + E[1 * np_ + p01])) / (2.0 * dx);
            double dEx_dy = ((E[0 * np_ + p01] + E[0 * np_ + p11]) - (E[0 * np_ + p00] + E[0 * np_ + p10])) / (2.0 * dy);
            int64_t o = (int64_t)j * nx + i;
            out[0 * cp + o] = dEz_dy;
            out[1 * cp + o] = -dEz_dx;
            out[2 * cp + o] = dEy_dx - dEx_dy;
        }
    }
}

/* Node value of a cell field: mean of the cells sharing the node (4 inside,
 * the 2 inside the box on a wall column). */
void orc_node_average(int nx, int ny, int periodic_x, const double *Hc, double *Bn)
{
    int nxn = node_cols(nx, periodic_x);
    int64_t cp = (int64_t)ny * nx, np_ = (int64_t)ny * nxn;
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < ny; ++j) {
            int jm = (j == 0) ? ny - 1 : j - 1;
            for (int i = 0; i < nxn; ++i) {
                double s;
                if (!periodic_x && (i == 0 || i == nx)) {
                    int ic = (i == 0) ? 0 : nx - 1;
                    s = 0.5 * (Hc[c * cp + (int64_t)j * nx + ic] + Hc[c * cp + (int64_t)jm * nx + ic]);
                } else {
                    int im = (i == 0) ? nx - 1 : i - 1;
                    s = 0.25 * (Hc[c * cp + (int64_t)j * nx + i] + Hc[c * cp + (int64_t)j * nx + im] +
                                Hc[c * cp + (int64_t)jm * nx + i] + Hc[c * cp + (int64_t)jm * nx + im]);
                }
                Bn[c * np_ + (int64_t)j * nxn + i] = s;
            }
        }
}

/* Solve A z = r for a 3x3 system by Gaussian elimination with partial pivoting. */
static void solve3(double A[3][3], double r[3], double z[3])
{
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int row = col + 1; row < 3; ++row)
            if (fabs(A[row][col]) > fabs(A[piv][col])) piv = row;
        if (piv != col) {
            for (int k = 0; k < 3; ++k) { double t = A[col][k]; A[col][k] = A[piv][k]; A[piv][k] = t; }
            double t = r[col]; r[col] = r[piv]; r[piv] = t;
        }
        for (int row = col + 1; row < 3; ++row) {
            double f = A[row][col] / A[col][col];
            for (int k = col; k < 3; ++k) A[row][k] -= f * A[col][k];
            r[row] -= f * r[col];
        }
    }
    for (int row = 2; row >= 0; --row) {
        double s = r[row];
        for (int k = row + 1; k < 3; ++k) s -= A[row][k] * z[k];
        z[row] = s / A[row][row];
    }
}

/* Incident laser waveform at x = 0 (reading of the missing source, Eq. 15):
 * a0 sin(omega t) exp(-2 ln2 (t - t0)^2 / tau^2) for t >= 0, zero before. */
double orc_laser(double t, double a0, double omega, double tau, double t0)
{
    if (t < 0.0 || a0 == 0.0) return 0.0;
    double env = (tau > 0.0) ? exp(-2.0 * log(2.0) * (t - t0) * (t - t0) / (tau * tau)) : 1.0;
    return a0 * sin(omega * t) * env;
}

/*
 * One field advance in the paper's own form (Eqs. 4 and 5):
 *   (I + S) E^{n+1} = (I - S) E^n + dt (curl H^{n+1/2} - dj)     at every node
 *   H^{n+3/2}       = H^{n+1/2} - dt curl E^{n+1}                at every cell
 * S and dj are the area-normalised moments (planes 1..12 of M).  On a wall
 * column (reading of the missing Eq. 14) the node is treated as vacuum: Ex
 * advances with the one-sided dHz/dy, and Ey, Ez follow a first-order Mur
 * condition on the outgoing field -- at x = 0 on the field minus the incident
 * plane wave (reading of the missing Eq. 15), which is then added back.
 * t_new is the time of E^{n+1}.
 */
void orc_field_literal(int nx, int ny, int periodic_x, double dx, double dy, double dt, double t_new,
                       double a0, double omega, double tau, double t0, int pol,
                       const double *E, const double *H, const double *M,
                       double *Enew, double *Hnew, double *work_nodes3)
{
    int nxn = node_cols(nx, periodic_x);
    int64_t np_ = (int64_t)ny * nxn, cp = (int64_t)ny * nx;
    double *curlH = work_nodes3;
    orc_curl_h(nx, ny, periodic_x, dx, dy, H, curlH);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nxn; ++i) {
            int64_t o = (int64_t)j * nxn + i;
            if (!periodic_x && (i == 0 || i == nx)) continue;
            double A[3][3], r[3], z[3];
            for (int row = 0; row < 3; ++row) {
                double s_e = 0.0;
                for (int col = 0; col < 3; ++col) {
                    double S = M[(1 + 3 * row + col) * np_ + o];
                    A[row][col] = (row == col ? 1.0 : 0.0) + S;
                    s_e += ((row == col ? 1.0 : 0.0) - S) * E[col * np_ + o];
                }
                r[row] = s_e + dt * (curlH[row * np_ + o] - M[(10 + row) * np_ + o]);
            }
            solve3(A, r, z);
            for (int c = 0; c < 3; ++c) Enew[c * np_ + o] = z[c];
        }
    if (!periodic_x) {
        double kap = (dt - dx) / (dt + dx);
        double t_old = t_new - dt;
        int pc = (pol == 0) ? 1 : 2; /* polarised component */
        for (int j = 0; j < ny; ++j) {
            /* x = 0 */
            int64_t o0 = (int64_t)j * nxn + 0, o1 = (int64_t)j * nxn + 1;
            Enew[0 * np_ + o0] = E[0 * np_ + o0] + dt * curlH[0 * np_ + o0];
            for (int c = 1; c < 3; ++c) {
                double inc_new0 = (c == pc) ? orc_laser(t_new, a0, omega, tau, t0) : 0.0;
                double inc_old0 = (c == pc) ? orc_laser(t_old, a0, omega, tau, t0) : 0.0;
                double inc_new1 = (c == pc) ? orc_laser(t_new - dx, a0, omega, tau, t0) : 0.0;
                double inc_old1 = (c == pc) ? orc_laser(t_old - dx, a0, omega, tau, t0) : 0.0;
                double s0_old = E[c * np_ + o0] - inc_old0;
                double s1_old = E[c * np_ + o1] - inc_old1;
                double s1_new = Enew[c * np_ + o1] - inc_new1;
                Enew[c * np_ + o0] = inc_new0 + s1_old + kap * (s1_new - s0_old);
            }
            /* x = Lx */
            int64_t oN = (int64_t)j * nxn + nx, oM = (int64_t)j * nxn + nx - 1;
            Enew[0 * np_ + oN] = E[0 * np_ + oN] + dt * curlH[0 * np_ + oN];
            for (int c = 1; c < 3; ++c)
                Enew[c * np_ + oN] = E[c * np_ + oM] + kap * (Enew[c * np_ + oM] - E[c * np_ + oN]);
        }
    }
    /* Eq. 5 */
    double *curlE = Hnew; /* reuse the output as scratch, then finish in place */
    orc_curl_e(nx, ny, periodic_x, dx, dy, Enew, curlE);
    for (int64_t k = 0; k < 3 * cp; ++k) Hnew[k] = H[k] - dt * curlE[k];
}
