// Field solve (Section 2, Eqs. 4-5; Section 3.3 steps 3-9 without the
// inter-processor messages): E at the nodes, H at the cell centres.
//
// literal mode: per node (I + S) E^{n+1} = (I - S) E^n + dt (curl_h H - dj)
//               with a closed-form 3x3 inverse, walls by a first-order Mur
//               condition and the incident plane wave at x = 0, then
//               H^{n+3/2} = H^{n+1/2} - dt curl_e E^{n+1}.
// CN mode:      (I + S) X + (dt/2)^2 curl_h curl_e X = E^n + (dt/2)(curl_h H^n - dj)
//               solved inside one cooperative kernel by FP64 iterative
//               refinement around an FP32 block-Jacobi BiCGSTAB, then
//               E^{n+1} = 2X - E^n, H^{n+1} = H^n - dt curl_e X.
// All kernels are bandwidth-bound stencils over node/cell arrays of V4.
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>

#include "pic_internal.cuh"

namespace cg = cooperative_groups;

namespace pic {

// Closed-form solution of A z = r (A 3x3) by the adjugate.
template <typename R>
__device__ inline void solve3(const R a[9], const R r[3], R z[3]) {
    R c00 = a[4] * a[8] - a[5] * a[7];
    R c01 = a[5] * a[6] - a[3] * a[8];
    R c02 = a[3] * a[7] - a[4] * a[6];
    R det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    R id = R(1) / det;
    z[0] = (c00 * r[0] + (a[2] * a[7] - a[1] * a[8]) * r[1] + (a[1] * a[5] - a[2] * a[4]) * r[2]) * id;
    z[1] = (c01 * r[0] + (a[0] * a[8] - a[2] * a[6]) * r[1] + (a[2] * a[3] - a[0] * a[5]) * r[2]) * id;
    z[2] = (c02 * r[0] + (a[1] * a[6] - a[0] * a[7]) * r[1] + (a[0] * a[4] - a[1] * a[3]) * r[2]) * id;
}

// curl_h of cell-centred H at interior node (i, j): centred differences over
// the four cells sharing the node (a = (i,j), b = (i-1,j), c = (i,j-1),
// d = (i-1,j-1)), averaged transversely.  With the diagonal differences
// p = a.z - d.z and q = b.z - c.z the two Hz derivatives are (p + q)/(2 dy)
// and (p - q)/(2 dx): returned are u = p + q, v = q - p, sy = 2 dx dHy/dx and
// sx = 2 dy dHx/dy (10 FP64 operations), so that
// curl_h H = (u/(2 dy), v/(2 dx), sy/(2 dx) - sx/(2 dy)).  The FP64 pipe, not
// memory, bounds the FP64 field kernels on this GPU.
template <typename R>
__device__ inline void curl_h_parts(const GridArgs<R> &g, const V4<R> *__restrict__ H, int i, int j, R &u, R &v, R &sy,
                                    R &sx) {
    int im = (i == 0) ? g.nx - 1 : i - 1;
    int jm = (j == 0) ? g.ny - 1 : j - 1;
    V4<R> a = H[(int64_t)j * g.nx + i], b = H[(int64_t)j * g.nx + im];
    V4<R> c = H[(int64_t)jm * g.nx + i], d = H[(int64_t)jm * g.nx + im];
    const R pz = a.z - d.z, qz = b.z - c.z;
    u = pz + qz;
    v = qz - pz;
    sy = (a.y - d.y) + (c.y - b.y);
    sx = (a.x - d.x) + (b.x - c.x);
}

// Node tiles of the touched-tile map (nullptr: every tile may hold moments).
// clr / clr_lo (or nullptr): the moment planes (and compensation planes)
// that the E solve zeroes on the touched tiles once it has read them, so that
// the next push deposits into cleared moments without a pass of its own.
template <typename R>
struct TouchArgs {
    const uint8_t *touched;
    int tnx, tny, ntx;
    R *clr, *clr_lo;
};

template <typename R>
__device__ inline void clear_node_moments(const GridArgs<R> &g, const TouchArgs<R> &tm, int64_t node) {
#pragma unroll
    for (int k = 0; k < NMOM; ++k) {
        tm.clr[(int64_t)k * g.nnode + node] = R(0);
        if (tm.clr_lo) tm.clr_lo[(int64_t)k * g.nnode + node] = R(0);
    }
}

template <typename R>
__global__ void k_field_E_literal(GridArgs<R> g, const V4<R> *__restrict__ E, const V4<R> *__restrict__ H,
                                  const R *M, const R *Mlo, V4<R> *__restrict__ Enew,
                                  V4<R> *__restrict__ Ehalf, TouchArgs<R> tm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nxn || j >= g.ny) return;
    const int64_t node = (int64_t)j * g.nxn + i;
    const bool touched = !tm.touched || tm.touched[(j / tm.tny) * tm.ntx + min(i / tm.tnx, tm.ntx - 1)];
    if (!g.periodic_x && (i == 0 || i == g.nx)) {   // wall columns: k_field_walls (their moments are not read)
        if (tm.clr && touched) clear_node_moments(g, tm, node);
        return;
    }
    R cu, cvv, sy, sx;
    curl_h_parts(g, H, i, j, cu, cvv, sy, sx);
    const R cx = cu * g.hy, cy = cvv * g.hx, cz = fma(sy, g.hx, -(sx * g.hy));
    V4<R> e = E[node];
    {
        if (!touched) {
            // vacuum (S = 0, dj = 0 on every node of the tile): Eq. 4 reduces to E^{n+1} = E^n + dt curl_h H,
            // with no moment read and no 3x3 solve.  The same operations as the solve below on such a node
            // (where the 3x3 solve returns its right-hand side exactly), so a node's bits do not depend on
            // whether its tile was marked.
            const R zx = fma(g.dt, cx, e.x), zy = fma(g.dt, cy, e.y), zz = fma(g.dt, cz, e.z);
            Enew[node] = V4<R>{zx, zy, zz, R(0)};
            Ehalf[pidx(g, i, j)] = V4<R>{R(0.5) * (e.x + zx), R(0.5) * (e.y + zy), R(0.5) * (e.z + zz), R(0)};
            return;
        }
    }
    R ia = g.inv_dx * g.inv_dy;
    R a[9], r[3], z[3];
    R ev[3] = {e.x, e.y, e.z};
    R cv[3] = {cx, cy, cz};
#pragma unroll
    for (int row = 0; row < 3; ++row) {
        R s_e = R(0);
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            const int64_t mi = (int64_t)(1 + 3 * row + col) * g.nnode + node;
            R S = (Mlo ? M[mi] + Mlo[mi] : M[mi]) * ia;
            a[3 * row + col] = (row == col ? R(1) : R(0)) + S;
            s_e += ((row == col ? R(1) : R(0)) - S) * ev[col];
        }
        const int64_t ji = (int64_t)(10 + row) * g.nnode + node;
        r[row] = fma(g.dt, cv[row] - (Mlo ? M[ji] + Mlo[ji] : M[ji]) * ia, s_e);
    }
    if (tm.clr) clear_node_moments(g, tm, node);   // read above by this thread only
    solve3(a, r, z);
    Enew[node] = V4<R>{z[0], z[1], z[2], R(0)};
    Ehalf[pidx(g, i, j)] = V4<R>{R(0.5) * (e.x + z[0]), R(0.5) * (e.y + z[1]), R(0.5) * (e.z + z[2]), R(0)};
}

struct Inc {
    double new0[3], old0[3], new1[3], old1[3];
};

// Wall columns (reading of the missing boundary and source equations): the wall
// node is vacuum; Ex advances with the one-sided dHz/dy, Ey and Ez follow a
// first-order Mur condition on the outgoing field -- at x = 0 on the field
// minus the incident wave, which is added back.
template <typename R>
__global__ void k_field_walls(GridArgs<R> g, const V4<R> *__restrict__ E, const V4<R> *__restrict__ H,
                              V4<R> *__restrict__ Enew, V4<R> *__restrict__ Ehalf, Inc inc, R kap) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= g.ny) return;
    int jm = (j == 0) ? g.ny - 1 : j - 1;
    {
        int64_t o0 = (int64_t)j * g.nxn, o1 = o0 + 1;
        V4<R> e0 = E[o0], e1 = E[o1], n1 = Enew[o1];
        R dhz = (H[(int64_t)j * g.nx].z - H[(int64_t)jm * g.nx].z) * g.inv_dy;
        V4<R> z;
        z.x = e0.x + g.dt * dhz;
        R s0y = e0.y - (R)inc.old0[1], s1y = e1.y - (R)inc.old1[1], n1y = n1.y - (R)inc.new1[1];
        R s0z = e0.z - (R)inc.old0[2], s1z = e1.z - (R)inc.old1[2], n1z = n1.z - (R)inc.new1[2];
        z.y = (R)inc.new0[1] + s1y + kap * (n1y - s0y);
        z.z = (R)inc.new0[2] + s1z + kap * (n1z - s0z);
        z.w = R(0);
        Enew[o0] = z;
        Ehalf[pidx(g, 0, j)] = V4<R>{R(0.5) * (e0.x + z.x), R(0.5) * (e0.y + z.y), R(0.5) * (e0.z + z.z), R(0)};
    }
    {
        int64_t oN = (int64_t)j * g.nxn + g.nx, oM = oN - 1;
        V4<R> eN = E[oN], eM = E[oM], nM = Enew[oM];
        R dhz = (H[(int64_t)j * g.nx + g.nx - 1].z - H[(int64_t)jm * g.nx + g.nx - 1].z) * g.inv_dy;
        V4<R> z;
        z.x = eN.x + g.dt * dhz;
        z.y = eM.y + kap * (nM.y - eN.y);
        z.z = eM.z + kap * (nM.z - eN.z);
        z.w = R(0);
        Enew[oN] = z;
        Ehalf[pidx(g, g.nx, j)] = V4<R>{R(0.5) * (eN.x + z.x), R(0.5) * (eN.y + z.y), R(0.5) * (eN.z + z.z), R(0)};
    }
}

// Eq. 5: H_out = H_in - dt curl_e(Ec), curl_e at the cell centre from its
// four corners (transversely averaged centred differences).  With the
// diagonal differences p = e11 - e00 and q = e01 - e10 the two Ez derivatives
// are (p + q)/(2 dy) and (p - q)/(2 dx); kx = dt/(2 dx), ky = dt/(2 dy) come
// from the host, so no thread divides (15 FP64 operations per cell).
template <typename R, typename RE>
__global__ void k_field_H(GridArgs<R> g, const V4<RE> *__restrict__ Ec, const V4<R> *__restrict__ Hin,
                          V4<R> *__restrict__ Hout, RE kx, RE ky) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    int ip = i + 1;
    if (g.periodic_x && ip == g.nx) ip = 0;
    int jp = (j + 1 == g.ny) ? 0 : j + 1;
    V4<RE> e00 = Ec[(int64_t)j * g.nxn + i], e10 = Ec[(int64_t)j * g.nxn + ip];
    V4<RE> e01 = Ec[(int64_t)jp * g.nxn + i], e11 = Ec[(int64_t)jp * g.nxn + ip];
    const RE pz = e11.z - e00.z, qz = e01.z - e10.z;
    const RE sy = (e11.y - e00.y) + (e10.y - e01.y);   // 2 dx dEy/dx
    const RE sx = (e11.x - e00.x) + (e01.x - e10.x);   // 2 dy dEx/dy
    int64_t o = (int64_t)j * g.nx + i;
    V4<R> hv = Hin[o];
    Hout[o] = V4<R>{(R)fma(-ky, pz + qz, (RE)hv.x), (R)fma(kx, pz - qz, (RE)hv.y),
                    (R)fma(ky, sx, fma(-kx, sy, (RE)hv.z)), R(0)};
}

// Node B: mean of the cells sharing the node (2 on a wall column).
template <typename R>
__global__ void k_node_average(GridArgs<R> g, const V4<R> *__restrict__ Hc, V4<R> *__restrict__ Bp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nxn || j >= g.ny) return;
    int jm = (j == 0) ? g.ny - 1 : j - 1;
    V4<R> o;
    if (!g.periodic_x && (i == 0 || i == g.nx)) {
        int ic = (i == 0) ? 0 : g.nx - 1;
        V4<R> a = Hc[(int64_t)j * g.nx + ic], b = Hc[(int64_t)jm * g.nx + ic];
        o = V4<R>{R(0.5) * (a.x + b.x), R(0.5) * (a.y + b.y), R(0.5) * (a.z + b.z), R(0)};
    } else {
        int im = (i == 0) ? g.nx - 1 : i - 1;
        V4<R> a = Hc[(int64_t)j * g.nx + i], b = Hc[(int64_t)j * g.nx + im];
        V4<R> c = Hc[(int64_t)jm * g.nx + i], d = Hc[(int64_t)jm * g.nx + im];
        o = V4<R>{R(0.25) * (a.x + b.x + c.x + d.x), R(0.25) * (a.y + b.y + c.y + d.y),
                  R(0.25) * (a.z + b.z + c.z + d.z), R(0)};
    }
    Bp[pidx(g, i, j)] = o;
}

// Ghost ring of a padded node array: periodic copies in y (and x when periodic),
// zero beyond a wall.  One thread per ring entry: the G rows above and below
// (full width), then the G columns left and right of every real row.
template <typename R>
__global__ void k_fill_ghosts(GridArgs<R> g, int nyp, V4<R> *__restrict__ F) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t band = (int64_t)g.G * g.nxp, side = (int64_t)g.ny * (g.nxp - g.nxn);
    if (t >= 2 * band + side) return;
    int pi, pj;
    if (t < band) {
        pj = (int)(t / g.nxp);
        pi = (int)(t - (int64_t)pj * g.nxp);
    } else if (t < 2 * band) {
        const int64_t u = t - band;
        pj = g.G + g.ny + (int)(u / g.nxp);
        pi = (int)(u % g.nxp);
    } else {
        const int64_t u = t - 2 * band;
        const int w = g.nxp - g.nxn;   // 2 G
        const int row = (int)(u / w), col = (int)(u - (int64_t)row * w);
        pj = g.G + row;
        pi = col < g.G ? col : g.nxn + col;
    }
    int i = pi - g.G, j = pj - g.G;
    int jj = ((j % g.ny) + g.ny) % g.ny;
    V4<R> v{R(0), R(0), R(0), R(0)};
    if (g.periodic_x) {
        int ii = ((i % g.nxn) + g.nxn) % g.nxn;
        v = F[pidx(g, ii, jj)];
    } else if (i >= 0 && i < g.nxn) {
        v = F[pidx(g, i, jj)];
    }
    F[(int64_t)pj * g.nxp + pi] = v;
}

// --------------------------------------------------------------------------- CN solver

// Mixed-precision solve.  The outer loop is iterative refinement in FP64:
// r = b - A x with FP64 moments and FP64 iterate, stop when |r| <= tol |b|;
// otherwise an FP32 block-Jacobi BiCGSTAB solves A d = r to a relative
// residual of CN_INNER_RTOL and x += d.  The FP32 operator differs from A
// by rounding (~1e-7 relative), far below 1/cond(A), so every refinement cuts
// the FP64 residual by about the inner tolerance.
struct CNVec {
    V4<double> *x, *b;                              // FP64 iterate and right-hand side
    V4<double> *cc;                                 // FP64 residual: curl_e x at the cells
    V4<float> *d, *r, *r0, *p, *v, *s, *t, *ph, *sh;  // FP32 inner solve of A d = r
    float *minv;                                    // [9][nnode] block-Jacobi inverse
    float *S;                                       // [9][nnode] S / dA
    // spectral preconditioner (nx, ny powers of two): complex work arrays of
    // nnode entries and twiddles e^{-2 pi i t / n}, t < n/2, for x and y
    float2 *FA, *FB, *GA, *GB, *twx, *twy;
    int fft, lx, ly;
    // line preconditioner (walls, ny a power of two): per column means of the
    // diagonal of S ([3][nxn]), the factors ([10][nxn][ny/2 + 1]) and the sweep
    // work ([6][nxn][ny/2 + 1]) of the per-mode block-tridiagonal solves
    float *scol, *lf, *lw;
    int line;
};

constexpr float CN_INNER_RTOL = 1e-4f;
constexpr int CN_MAX_OUTER = 30;

// A box with walls (the wall node is vacuum): the x row is X_x + (dt/2)^2
// (curl_h curl_e X)_x with the wall column's one-sided curl_h, i.e.
// 2 hy (Cz(ic, j) - Cz(ic, j-1)) of the inside cell column ic; the y and z
// rows are the time-centred Mur condition cw X_w + cv X_v (v the neighbour
// column, cw = 1/dt + 1/dx, cv = 1/dt - 1/dx).
struct WallRows {
    double cw, cv;
};

template <typename T>
__device__ inline T cell_curl_z(const V4<T> &e00, const V4<T> &e10, const V4<T> &e01, const V4<T> &e11, T hx, T hy) {
    return ((e10.y + e11.y) - (e00.y + e01.y)) * hx - ((e01.x + e11.x) - (e00.x + e10.x)) * hy;
}

template <typename T>
__device__ inline V4<T> apply_A_wall(const GridArgs<double> &g, const V4<T> *__restrict__ X, T c2, T hx, T hy, T cw,
                                     T cv, int i, int j) {
    const int ic = (i == 0) ? 0 : g.nx - 1, iv = (i == 0) ? 1 : g.nx - 1;
    const int jm = (j == 0) ? g.ny - 1 : j - 1, jp = (j + 1 == g.ny) ? 0 : j + 1;
    auto at = [&](int a, int b) { return X[(int64_t)b * g.nxn + a]; };
    const V4<T> m0 = at(ic, jm), m1 = at(ic + 1, jm), c0 = at(ic, j), c1 = at(ic + 1, j), p0 = at(ic, jp),
                p1 = at(ic + 1, jp);
    const T up = cell_curl_z(c0, c1, p0, p1, hx, hy), dn = cell_curl_z(m0, m1, c0, c1, hx, hy);
    const V4<T> xw = at(i, j), xv = at(iv, j);
    return V4<T>{xw.x + c2 * ((up - dn) * (T(2) * hy)), cw * xw.y + cv * xv.y, cw * xw.z + cv * xv.z, T(0)};
}

// (I + S) X + (dt/2)^2 curl_h curl_e X at node (i, j) (wall nodes: apply_A_wall);
// S9 points at the 9 planar S rows (stride nnode), each scaled by sc.
template <typename T>
__device__ inline V4<T> apply_A(const GridArgs<double> &g, const V4<T> *__restrict__ X, const T *__restrict__ S9,
                                T sc, T c2, T hx, T hy, int i, int j, T cw = T(0), T cv = T(0)) {
    if (!g.periodic_x && (i == 0 || i == g.nx)) return apply_A_wall<T>(g, X, c2, hx, hy, cw, cv, i, j);
    int im = (i == 0) ? g.nx - 1 : i - 1, ip = (g.periodic_x && i + 1 == g.nx) ? 0 : i + 1;
    int jm = (j == 0) ? g.ny - 1 : j - 1, jp = (j + 1 == g.ny) ? 0 : j + 1;
    const int xs[3] = {im, i, ip};
    const int ys[3] = {jm, j, jp};
    V4<T> n[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) n[b][a] = X[(int64_t)ys[b] * g.nxn + xs[a]];
    // curl_e at the four cells around the node; cell (ci, cj) has corners n[cj][ci..ci+1], n[cj+1][...]
    T Cx[2][2], Cy[2][2], Cz[2][2];
#pragma unroll
    for (int cj = 0; cj < 2; ++cj)
#pragma unroll
        for (int ci = 0; ci < 2; ++ci) {
            const V4<T> &e00 = n[cj][ci], &e10 = n[cj][ci + 1], &e01 = n[cj + 1][ci], &e11 = n[cj + 1][ci + 1];
            T dEz_dy = ((e01.z + e11.z) - (e00.z + e10.z)) * hy;
            T dEz_dx = ((e10.z + e11.z) - (e00.z + e01.z)) * hx;
            T dEy_dx = ((e10.y + e11.y) - (e00.y + e01.y)) * hx;
            T dEx_dy = ((e01.x + e11.x) - (e00.x + e10.x)) * hy;
            Cx[cj][ci] = dEz_dy;
            Cy[cj][ci] = -dEz_dx;
            Cz[cj][ci] = dEy_dx - dEx_dy;
        }
    // curl_h at the node from cells a = [1][1], b = [1][0], c = [0][1], d = [0][0]
    T kx = ((Cz[1][1] + Cz[1][0]) - (Cz[0][1] + Cz[0][0])) * hy;
    T ky = -(((Cz[1][1] + Cz[0][1]) - (Cz[1][0] + Cz[0][0])) * hx);
    T kz = ((Cy[1][1] + Cy[0][1]) - (Cy[1][0] + Cy[0][0])) * hx - ((Cx[1][1] + Cx[1][0]) - (Cx[0][1] + Cx[0][0])) * hy;
    int64_t node = (int64_t)j * g.nxn + i;
    const V4<T> &xc = n[1][1];
    T S[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) S[k] = S9[(int64_t)k * g.nnode + node] * sc;
    V4<T> y;
    y.x = xc.x + (S[0] * xc.x + S[1] * xc.y + S[2] * xc.z) + c2 * kx;
    y.y = xc.y + (S[3] * xc.x + S[4] * xc.y + S[5] * xc.z) + c2 * ky;
    y.z = xc.z + (S[6] * xc.x + S[7] * xc.y + S[8] * xc.z) + c2 * kz;
    y.w = T(0);
    return y;
}

// The FP64 residual's operator in two passes, with the expressions of
// apply_A: curl_e of X once per cell (cell (ci, cj) has corners (ci, cj),
// (ci+1, cj), (ci, cj+1), (ci+1, cj+1), periodic), then per node curl_h of
// those cell values, S X and X.  Each cell's curl is computed once instead of
// once for each of its four corner nodes; the results are the same bits.
__device__ inline V4<double> cell_curl_e(const GridArgs<double> &g, const V4<double> *__restrict__ X, double hx,
                                         double hy, int ci, int cj) {
    const int ip = (g.periodic_x && ci + 1 == g.nx) ? 0 : ci + 1, jp = (cj + 1 == g.ny) ? 0 : cj + 1;
    const V4<double> e00 = X[(int64_t)cj * g.nxn + ci], e10 = X[(int64_t)cj * g.nxn + ip];
    const V4<double> e01 = X[(int64_t)jp * g.nxn + ci], e11 = X[(int64_t)jp * g.nxn + ip];
    const double dEz_dy = ((e01.z + e11.z) - (e00.z + e10.z)) * hy;
    const double dEz_dx = ((e10.z + e11.z) - (e00.z + e01.z)) * hx;
    const double dEy_dx = ((e10.y + e11.y) - (e00.y + e01.y)) * hx;
    const double dEx_dy = ((e01.x + e11.x) - (e00.x + e10.x)) * hy;
    return V4<double>{dEz_dy, -dEz_dx, dEy_dx - dEx_dy, 0.0};
}

__device__ inline V4<double> apply_A_from_cells(const GridArgs<double> &g, const V4<double> *__restrict__ X,
                                                const V4<double> *__restrict__ Cc, const double *__restrict__ S9,
                                                double sc, double c2, double hx, double hy, int i, int j,
                                                double cw = 0.0, double cv = 0.0) {
    const int im = (i == 0) ? g.nx - 1 : i - 1, jm = (j == 0) ? g.ny - 1 : j - 1;
    if (!g.periodic_x && (i == 0 || i == g.nx)) {   // wall node (apply_A_wall with the cells' curls)
        const int ic = (i == 0) ? 0 : g.nx - 1, iv = (i == 0) ? 1 : g.nx - 1;
        const double up = Cc[(int64_t)j * g.nx + ic].z, dn = Cc[(int64_t)jm * g.nx + ic].z;
        const V4<double> xw = X[(int64_t)j * g.nxn + i], xv = X[(int64_t)j * g.nxn + iv];
        return V4<double>{xw.x + c2 * ((up - dn) * (2.0 * hy)), cw * xw.y + cv * xv.y, cw * xw.z + cv * xv.z, 0.0};
    }
    // cells a = [1][1] (i, j), b = [1][0] (im, j), c = [0][1] (i, jm), d = [0][0] (im, jm)
    const V4<double> c11 = Cc[(int64_t)j * g.nx + i], c10 = Cc[(int64_t)j * g.nx + im];
    const V4<double> c01 = Cc[(int64_t)jm * g.nx + i], c00 = Cc[(int64_t)jm * g.nx + im];
    const double kx = ((c11.z + c10.z) - (c01.z + c00.z)) * hy;
    const double ky = -(((c11.z + c01.z) - (c10.z + c00.z)) * hx);
    const double kz = ((c11.y + c01.y) - (c10.y + c00.y)) * hx - ((c11.x + c10.x) - (c01.x + c00.x)) * hy;
    const int64_t node = (int64_t)j * g.nxn + i;
    const V4<double> xc = X[node];
    double S[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) S[k] = S9[(int64_t)k * g.nnode + node] * sc;
    V4<double> y;
    y.x = xc.x + (S[0] * xc.x + S[1] * xc.y + S[2] * xc.z) + c2 * kx;
    y.y = xc.y + (S[3] * xc.x + S[4] * xc.y + S[5] * xc.z) + c2 * ky;
    y.z = xc.z + (S[6] * xc.x + S[7] * xc.y + S[8] * xc.z) + c2 * kz;
    y.w = 0.0;
    return y;
}

__device__ inline V4<float> apply_minv(const float *__restrict__ mi, int64_t nnode, int64_t node, const V4<float> &v) {
    float a[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) a[k] = mi[(int64_t)k * nnode + node];
    return V4<float>{a[0] * v.x + a[1] * v.y + a[2] * v.z, a[3] * v.x + a[4] * v.y + a[5] * v.z,
                     a[6] * v.x + a[7] * v.y + a[8] * v.z, 0.f};
}

template <typename T>
__device__ inline T dot(const V4<T> &a, const V4<T> &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// ---- spectral preconditioner ------------------------------------------------
// On a periodic grid the operator (1 + s) X + c2 curl_h curl_e X with a
// uniform s is diagonal in Fourier space: for the mode e^{i(a i + b j)}, with
// p = (e^{ia} - 1)(1 + e^{ib}) / (2 dx) and q = (1 + e^{ia})(e^{ib} - 1) / (2 dy)
// (the symbols of d/dx and d/dy from nodes to cells), curl_h curl_e acts as
// [[|q|^2, -q* p, 0], [-p* q, |p|^2, 0], [0, 0, |p|^2 + |q|^2]].  The
// preconditioner solves that 3x3 system per mode with s = the grid mean of the
// diagonal of S, using FP32 radix-2 FFTs along rows, a transpose, and FFTs
// along the other axis; x and y share one complex transform (x + i y).

__device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// In-place FFT of nrows rows of n = 2^logn complex values (row r of the
// first nrows_a rows in A, the rest in B), by the Stockham autosort form of
// the radix-2 transform: stage L = 1, 2, ..., n/2 reads x[j] and x[j + n/2]
// (j = q L + k < n/2) and writes y[2 q L + k] = x[j] + w^k x[j + n/2],
// y[2 q L + k + L] = x[j] - w^k x[j + n/2] with w = e^{-+2 pi i / (2L)},
// between two shared buffers.  Input and output are in natural order (no bit
// reversal), the reads are contiguous, and stage L takes its L twiddles from a
// table of its own (entries L - 1 ... 2L - 2), so that neighbouring threads
// read neighbouring words.  Short rows are transformed several at a time (up
// to FFT_GROUP values, at most the block's share of the rows), so that the
// threads have work between two barriers.  With vin the rows are read from
// a V4 vector instead (A rows: x + i y, B rows: z), with vout written to one
// (A rows give x, y and the spare component, B rows z).
constexpr int FFT_GROUP = 2048;

__device__ inline void fft_rows(float2 *A, float2 *B, int nrows_a, int n, int logn, const float2 *__restrict__ tw,
                                bool inverse, float2 *sm, const V4<float> *vin = nullptr,
                                V4<float> *vout = nullptr) {
    const int G = n > FFT_GROUP ? n : FFT_GROUP;
    float2 *buf0 = sm, *buf1 = sm + G, *tws = sm + 2 * G;
    const int nh = n >> 1;
    for (int t = threadIdx.x; t < n - 1; t += blockDim.x) {
        const int lg = 31 - __clz(t + 1), L = 1 << lg, k = t - (L - 1);   // stage L, twiddle k < L
        float2 w = tw[k * (nh >> lg)];
        if (inverse) w.y = -w.y;
        tws[t] = w;
    }
    __syncthreads();
    const int nrows = 2 * nrows_a;
    const int share = (nrows + gridDim.x - 1) / gridDim.x;
    const int rpb = max(1, min(G >> logn, share));
    for (int row0 = blockIdx.x * rpb; row0 < nrows; row0 += gridDim.x * rpb) {
        const int nr = min(rpb, nrows - row0);
        for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
            const int r = e >> logn, row = row0 + r;
            if (vin) {
                const bool a = row < nrows_a;
                const V4<float> q = vin[(int64_t)(a ? row : row - nrows_a) * n + (e & (n - 1))];
                buf0[e] = a ? make_float2(q.x, q.y) : make_float2(q.z, 0.f);
            } else {
                const float2 *d = row < nrows_a ? A + (int64_t)row * n : B + (int64_t)(row - nrows_a) * n;
                buf0[e] = d[e & (n - 1)];
            }
        }
        __syncthreads();
        float2 *x = buf0, *y = buf1;
        for (int lg = 0; lg < logn; ++lg) {
            const int L = 1 << lg;
            if (nr == 1) {   // one long row: no row index
                for (int j = threadIdx.x; j < nh; j += blockDim.x) {
                    const int k = j & (L - 1), o = ((j >> lg) << (lg + 1)) + k;
                    const float2 a = x[j], t = cmul(tws[L - 1 + k], x[j + nh]);
                    y[o] = make_float2(a.x + t.x, a.y + t.y);
                    y[o + L] = make_float2(a.x - t.x, a.y - t.y);
                }
            } else {
                for (int e = threadIdx.x; e < nr * nh; e += blockDim.x) {
                    const int r = e >> (logn - 1), j = e & (nh - 1);
                    const int k = j & (L - 1), o = r * n + ((j >> lg) << (lg + 1)) + k;
                    const float2 a = x[r * n + j], t = cmul(tws[L - 1 + k], x[r * n + j + nh]);
                    y[o] = make_float2(a.x + t.x, a.y + t.y);
                    y[o + L] = make_float2(a.x - t.x, a.y - t.y);
                }
            }
            __syncthreads();
            float2 *z = x;
            x = y;
            y = z;
        }
        for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
            const int r = e >> logn, row = row0 + r;
            if (vout) {
                V4<float> &q = vout[(int64_t)(row < nrows_a ? row : row - nrows_a) * n + (e & (n - 1))];
                if (row < nrows_a) {
                    q.x = x[e].x;
                    q.y = x[e].y;
                    q.w = 0.f;
                } else {
                    q.z = x[e].x;
                }
            } else {
                float2 *d = row < nrows_a ? A + (int64_t)row * n : B + (int64_t)(row - nrows_a) * n;
                d[e & (n - 1)] = x[e];
            }
        }
        __syncthreads();
    }
}

// out_a = in_a^T, out_b = in_b^T for R x C row-major arrays (32 x 32 tiles).
__device__ inline void transpose2(const float2 *in_a, const float2 *in_b, float2 *out_a, float2 *out_b, int R, int C,
                                  float2 *sm) {
    const int tr_n = (R + 31) / 32, tc_n = (C + 31) / 32, ntile = tr_n * tc_n;
    for (int tile = blockIdx.x; tile < 2 * ntile; tile += gridDim.x) {
        const float2 *in = tile < ntile ? in_a : in_b;
        float2 *out = tile < ntile ? out_a : out_b;
        const int tt = tile < ntile ? tile : tile - ntile;
        const int tr = tt / tc_n, tc = tt - tr * tc_n;
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int ty = e >> 5, tx = e & 31, r = tr * 32 + ty, c = tc * 32 + tx;
            if (r < R && c < C) sm[ty * 33 + tx] = in[(int64_t)r * C + c];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int ty = e >> 5, tx = e & 31, c = tc * 32 + ty, r = tr * 32 + tx;
            if (r < R && c < C) out[(int64_t)c * R + r] = sm[tx * 33 + ty];
        }
        __syncthreads();
    }
}

// out = P^{-1} in (all blocks of the cooperative grid take part; ends with out written).
__device__ inline void apply_spectral(cg::grid_group &grid, const GridArgs<double> &g, const CNVec &v,
                                      const V4<float> *in, V4<float> *out, float c2, float sx, float sy, float sz,
                                      float2 *sm) {
    const int nx = g.nx, ny = g.ny;
    const int64_t N = (int64_t)nx * ny;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    fft_rows(v.FA, v.FB, ny, nx, v.lx, v.twx, false, sm, in);    // along x: [y][x] (from in: x + i y, z)
    grid.sync();
    transpose2(v.FA, v.FB, v.GA, v.GB, ny, nx, sm);               // -> [x][y]
    grid.sync();
    fft_rows(v.GA, v.GB, nx, ny, v.ly, v.twy, false, sm);        // along y: spectra [kx][ky]
    grid.sync();
    const float ihx = 0.5f * (float)g.inv_dx, ihy = 0.5f * (float)g.inv_dy, inv_n = 1.f / (float)N;
    for (int64_t idx = tid; idx < N; idx += stride) {
        const int kx = (int)(idx / ny), ky = (int)(idx - (int64_t)kx * ny);
        const int64_t m = (int64_t)((nx - kx) & (nx - 1)) * ny + ((ny - ky) & (ny - 1));
        const float2 F = v.GA[idx], Fm = v.GA[m], Z = v.GB[idx];
        // X = (F + conj(Fm)) / 2, Y = (F - conj(Fm)) / (2i)
        const float2 X = make_float2(0.5f * (F.x + Fm.x), 0.5f * (F.y - Fm.y));
        const float2 Y = make_float2(0.5f * (F.y + Fm.y), -0.5f * (F.x - Fm.x));
        float sa, ca, sb, cb;
        sincospif(2.f * (float)kx / (float)nx, &sa, &ca);
        sincospif(2.f * (float)ky / (float)ny, &sb, &cb);
        // p = (e^{ia} - 1)(1 + e^{ib}) / (2 dx), q = (1 + e^{ia})(e^{ib} - 1) / (2 dy)
        const float2 ea1 = make_float2(ca - 1.f, sa), eb1 = make_float2(cb - 1.f, sb);
        const float2 ea2 = make_float2(ca + 1.f, sa), eb2 = make_float2(cb + 1.f, sb);
        float2 p = cmul(ea1, eb2), q = cmul(ea2, eb1);
        p = make_float2(p.x * ihx, p.y * ihx);
        q = make_float2(q.x * ihy, q.y * ihy);
        const float pp = p.x * p.x + p.y * p.y, qq = q.x * q.x + q.y * q.y;
        const float2 cqp = cmul(make_float2(q.x, -q.y), p);   // conj(q) p
        const float A11 = 1.f + sx + c2 * qq, A22 = 1.f + sy + c2 * pp;
        const float2 A12 = make_float2(-c2 * cqp.x, -c2 * cqp.y), A21 = make_float2(A12.x, -A12.y);
        const float idet = inv_n / (A11 * A22 - (A12.x * A12.x + A12.y * A12.y));
        const float2 a12y = cmul(A12, Y), a21x = cmul(A21, X);
        const float2 Xs = make_float2((A22 * X.x - a12y.x) * idet, (A22 * X.y - a12y.y) * idet);
        const float2 Ys = make_float2((A11 * Y.x - a21x.x) * idet, (A11 * Y.y - a21x.y) * idet);
        const float iz = inv_n / (1.f + sz + c2 * (pp + qq));
        v.FA[idx] = make_float2(Xs.x - Ys.y, Xs.y + Ys.x);   // X' + i Y'
        v.FB[idx] = make_float2(Z.x * iz, Z.y * iz);
    }
    grid.sync();
    fft_rows(v.FA, v.FB, nx, ny, v.ly, v.twy, true, sm);         // back along y: [kx][y]
    grid.sync();
    transpose2(v.FA, v.FB, v.GA, v.GB, nx, ny, sm);               // -> [y][kx]
    grid.sync();
    fft_rows(v.GA, v.GB, ny, nx, v.lx, v.twx, true, sm, nullptr, out);   // back along x: [y][x], into out
}

// ---- line preconditioner (walls) -----------------------------------------
// In a box with walls x is not periodic, y is.  For the y-mode e^{i b j}
// (j the node row) the operator (1 + s_i) X + c2 curl_h curl_e X couples a
// node column only to its two neighbours.  With ax = 1/(2 dx), ay = 1/(2 dy),
// A = 4 ay^2 sin^2(b/2), B = 4 ax^2 cos^2(b/2), sg = 2 ax ay sin b and
// Yt = i Y, the interior rows are real:
//   X:  (1 + sx_i + 2 c2 A) X_i + c2 A (X_{i-1} + X_{i+1}) + c2 sg (Yt_{i+1} - Yt_{i-1})
//   Yt: (1 + sy_i + 2 c2 B) Yt_i - c2 B (Yt_{i-1} + Yt_{i+1}) - c2 sg (X_{i+1} - X_{i-1})
//   Z:  (1 + sz_i + 2 c2 (A + B)) Z_i + c2 (A - B) (Z_{i-1} + Z_{i+1})
// and the wall rows (vacuum, the one-sided curl_h of the inside cell column,
// the time-centred Mur condition) are, at i = 0 (v = 1; at i = nx, v = nx - 1
// and the sign of the sg terms flipped):
//   X:  (1 + 2 c2 A) X_w + 2 c2 A X_v - 2 c2 sg (Yt_w - Yt_v),  Yt: cw Yt_w + cv Yt_v,  Z: cw Z_w + cv Z_v.
// s_i = the mean over the column of the diagonal of S (0 on the walls).  The
// preconditioner solves these block-tridiagonal systems exactly, mode by mode
// (block Thomas, factored once per solve): FP32 FFTs along y of x + i y and
// z, one thread per mode b = 0 .. ny/2 sweeping the columns (the modes -b are
// the conjugates: the fields are real), and the inverse FFTs.  Without a
// plasma (S = 0) it inverts the vacuum operator.
struct LineCoef {
    float A, B, sg;
};

__device__ inline LineCoef line_coef(const GridArgs<double> &g, int b) {
    float sn, cs, sh, ch;
    sincospif((float)b / (float)g.ny, &sh, &ch);          // b/2 of the mode angle 2 pi b / ny
    sincospif(2.f * (float)b / (float)g.ny, &sn, &cs);
    const float ax = 0.5f * (float)g.inv_dx, ay = 0.5f * (float)g.inv_dy;
    return LineCoef{4.f * ay * ay * sh * sh, 4.f * ax * ax * ch * ch, 2.f * ax * ay * sn};
}

// The 2 x 2 (X, Yt) blocks of row i: diagonal D, left L (column i - 1), right U (column i + 1).
__device__ inline void line_blocks(const GridArgs<double> &g, const LineCoef &k, float c2, float cw, float cv,
                                   const float *scol, int i, float (&D)[4], float (&L)[4], float (&U)[4], float &dz,
                                   float &lz, float &uz) {
    const int nxn = g.nxn;
    const float a = c2 * k.A, bb = c2 * k.B, s = c2 * k.sg;
    if (i == 0 || i == g.nx) {
        const float sgn = (i == 0) ? 1.f : -1.f;   // Yt_w - Yt_v at x = 0, the opposite at x = Lx
        const float D_[4] = {1.f + 2.f * a, -2.f * s * sgn, 0.f, cw};
        const float O_[4] = {2.f * a, 2.f * s * sgn, 0.f, cv};
        const float Z_[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < 4; ++q) {
            D[q] = D_[q];
            L[q] = (i == 0) ? Z_[q] : O_[q];
            U[q] = (i == 0) ? O_[q] : Z_[q];
        }
        dz = cw;
        lz = (i == 0) ? 0.f : cv;
        uz = (i == 0) ? cv : 0.f;
        return;
    }
    D[0] = 1.f + scol[i] + 2.f * a;
    D[1] = 0.f;
    D[2] = 0.f;
    D[3] = 1.f + scol[nxn + i] + 2.f * bb;
    L[0] = a;  L[1] = -s; L[2] = s;  L[3] = -bb;
    U[0] = a;  U[1] = s;  U[2] = -s; U[3] = -bb;
    dz = 1.f + scol[2 * nxn + i] + 2.f * (a + bb);
    lz = uz = a - bb;
}

__device__ inline void inv2(const float (&m)[4], float (&o)[4]) {
    const float id = 1.f / (m[0] * m[3] - m[1] * m[2]);
    o[0] = m[3] * id;
    o[1] = -m[1] * id;
    o[2] = -m[2] * id;
    o[3] = m[0] * id;
}

__device__ inline void mul2(const float (&p)[4], const float (&q)[4], float (&o)[4]) {
    o[0] = p[0] * q[0] + p[1] * q[2];
    o[1] = p[0] * q[1] + p[1] * q[3];
    o[2] = p[2] * q[0] + p[3] * q[2];
    o[3] = p[2] * q[1] + p[3] * q[3];
}

// Per-column means of the diagonal of S, then the factors of every mode: for
// column i, Dp_i = D_i - M_i U_{i-1} with M_i = L_i Dp_{i-1}^{-1}; stored, mode
// by mode (lf[b][q][i]), are Dp_i^{-1} (q = 0..3), M_i (4..7), 1/dp_i and m_i
// of the Z row (8, 9).  nbm = ny/2 + 1 modes.
__device__ inline void line_setup(cg::grid_group &grid, const GridArgs<double> &g, const CNVec &v, float c2, float cw,
                                  float cv) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int nxn = g.nxn, nbm = g.ny / 2 + 1;
    const int64_t N = g.nnode;
    for (int64_t i = tid; i < nxn; i += stride) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        if (i != 0 && i != g.nx)
            for (int j = 0; j < g.ny; ++j) {
                const int64_t n = (int64_t)j * nxn + i;
                a0 += v.S[n];
                a1 += v.S[4 * N + n];
                a2 += v.S[8 * N + n];
            }
        const float inv = 1.f / (float)g.ny;
        v.scol[i] = a0 * inv;
        v.scol[nxn + i] = a1 * inv;
        v.scol[2 * nxn + i] = a2 * inv;
    }
    const int hyn = g.ny / 2;
    for (int64_t t = tid; t < hyn; t += stride) {
        double sn, cs;
        sincospi(-2.0 * (double)t / g.ny, &sn, &cs);
        v.twy[t] = make_float2((float)cs, (float)sn);
    }
    grid.sync();
    for (int64_t b = tid; b < nbm; b += stride) {
        const LineCoef k = line_coef(g, (int)b);
        float *lf = v.lf + b * 10 * (int64_t)nxn;
        float Dp[4], Dpi[4], Up[4], dpz = 0.f, upz = 0.f;
        for (int i = 0; i < nxn; ++i) {
            float D[4], L[4], U[4], dz, lz, uz, M[4] = {0.f, 0.f, 0.f, 0.f}, mz = 0.f;
            line_blocks(g, k, c2, cw, cv, v.scol, i, D, L, U, dz, lz, uz);
            if (i > 0) {
                mul2(L, Dpi, M);
                float MU[4];
                mul2(M, Up, MU);
                for (int q = 0; q < 4; ++q) Dp[q] = D[q] - MU[q];
                mz = lz / dpz;
                dpz = dz - mz * upz;
            } else {
                for (int q = 0; q < 4; ++q) Dp[q] = D[q];
                dpz = dz;
            }
            inv2(Dp, Dpi);
            for (int q = 0; q < 4; ++q) lf[q * nxn + i] = Dpi[q];
            for (int q = 0; q < 4; ++q) lf[(4 + q) * nxn + i] = M[q];
            lf[8 * nxn + i] = 1.f / dpz;
            lf[9 * nxn + i] = mz;
            for (int q = 0; q < 4; ++q) Up[q] = U[q];
            upz = uz;
        }
    }
}

// Shared memory of one mode's sweep: the mode's factors and the 6 right-hand-
// side and solution streams (3 complex values per column).
__host__ __device__ inline size_t line_sweep_bytes(int nxn) { return (size_t)nxn * 16 * sizeof(float); }

// out = P^{-1} in (all blocks of the cooperative grid take part; ends with out written).
__device__ inline void apply_line(cg::grid_group &grid, const GridArgs<double> &g, const CNVec &v,
                                  const V4<float> *in, V4<float> *out, float c2, float cw, float cv, float2 *sm) {
    const int nxn = g.nxn, ny = g.ny, nbm = ny / 2 + 1;
    const int64_t N = g.nnode;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    // columns as rows: GA[i][j] = x + i y, GB[i][j] = z
    for (int64_t e = tid; e < N; e += stride) {
        const int i = (int)(e / ny), j = (int)(e - (int64_t)i * ny);
        const V4<float> q = in[(int64_t)j * nxn + i];
        v.GA[e] = make_float2(q.x, q.y);
        v.GB[e] = make_float2(q.z, 0.f);
    }
    grid.sync();
    fft_rows(v.GA, v.GB, nxn, ny, v.ly, v.twy, false, sm);   // along y: [column][mode]
    grid.sync();
    transpose2(v.GA, v.GB, v.FA, v.FB, nxn, ny, sm);           // -> [mode][column]
    grid.sync();
    const float inv_n = 1.f / (float)ny;
    float *s_lf = (float *)sm;                 // [10][nxn]
    float *s_xr = s_lf + 10 * (size_t)nxn;     // (X, Yt) real parts, interleaved [nxn][2]
    float *s_xi = s_xr + 2 * (size_t)nxn;      // (X, Yt) imaginary parts
    float *s_zr = s_xi + 2 * (size_t)nxn, *s_zi = s_zr + nxn;
    for (int b = blockIdx.x; b < nbm; b += gridDim.x) {
        const int bm = (ny - b) & (ny - 1);
        const LineCoef k = line_coef(g, b);
        const float *lf = v.lf + (int64_t)b * 10 * nxn;
        for (int e = threadIdx.x; e < 10 * nxn; e += blockDim.x) s_lf[e] = lf[e];
        for (int i = threadIdx.x; i < nxn; i += blockDim.x) {
            const float2 F = v.FA[(int64_t)b * nxn + i], Fm = v.FA[(int64_t)bm * nxn + i], Z = v.FB[(int64_t)b * nxn + i];
            const float Xr = 0.5f * (F.x + Fm.x), Xi = 0.5f * (F.y - Fm.y);       // X_b = (F + conj(Fm)) / 2
            const float Yr = 0.5f * (F.y + Fm.y), Yi = -0.5f * (F.x - Fm.x);      // Y_b = (F - conj(Fm)) / (2i)
            s_xr[2 * i] = Xr;                                                      // (X, i Y): real parts
            s_xr[2 * i + 1] = -Yi;
            s_xi[2 * i] = Xi;                                                      // imaginary parts
            s_xi[2 * i + 1] = Yr;
            s_zr[i] = Z.x;
            s_zi[i] = Z.y;
        }
        __syncthreads();
        // four independent recurrences: (X, Yt) real and imaginary parts (threads 0, 1), Z real and
        // imaginary parts (threads 32, 33: another warp, so that the two kinds do not diverge in one)
        const int t = threadIdx.x;
        if (t < 2) {
            float *x = t == 0 ? s_xr : s_xi;
            float y0 = 0.f, y1 = 0.f;
            for (int i = 0; i < nxn; ++i) {   // y_i = r_i - M_i y_{i-1}
                float r0 = x[2 * i], r1 = x[2 * i + 1];
                if (i > 0) {
                    r0 -= s_lf[4 * nxn + i] * y0 + s_lf[5 * nxn + i] * y1;
                    r1 -= s_lf[6 * nxn + i] * y0 + s_lf[7 * nxn + i] * y1;
                }
                y0 = r0;
                y1 = r1;
                x[2 * i] = y0;
                x[2 * i + 1] = y1;
            }
            float x0 = 0.f, x1 = 0.f;
            for (int i = nxn - 1; i >= 0; --i) {   // x_i = Dp_i^{-1} (y_i - U_i x_{i+1})
                float t0 = x[2 * i], t1 = x[2 * i + 1];
                if (i < nxn - 1) {
                    float D[4], L[4], U[4], dz, lz, uz;
                    line_blocks(g, k, c2, cw, cv, v.scol, i, D, L, U, dz, lz, uz);
                    t0 -= U[0] * x0 + U[1] * x1;
                    t1 -= U[2] * x0 + U[3] * x1;
                }
                x0 = s_lf[i] * t0 + s_lf[nxn + i] * t1;
                x1 = s_lf[2 * nxn + i] * t0 + s_lf[3 * nxn + i] * t1;
                x[2 * i] = x0;
                x[2 * i + 1] = x1;
            }
        } else if (t == 32 || t == 33) {
            float *z = t == 32 ? s_zr : s_zi;
            float y = 0.f;
            for (int i = 0; i < nxn; ++i) {
                float r = z[i];
                if (i > 0) r -= s_lf[9 * nxn + i] * y;
                y = r;
                z[i] = y;
            }
            const float uz = c2 * (k.A - k.B);
            float xz = 0.f;
            for (int i = nxn - 1; i >= 0; --i) {
                float t = z[i];
                if (i < nxn - 1) t -= ((i == 0) ? cv : uz) * xz;   // row 0: the wall's Mur coefficient
                xz = s_lf[8 * nxn + i] * t;
                z[i] = xz;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nxn; i += blockDim.x) {
            // X' = xr[0] + i xi[0]; i Y' = xr[1] + i xi[1], so Y' = xi[1] - i xr[1]
            const float Xr = s_xr[2 * i], Xi = s_xi[2 * i], Yr = s_xi[2 * i + 1], Yi = -s_xr[2 * i + 1];
            const float zr = s_zr[i], zi = s_zi[i];
            // F' = X' + i Y' (mode b), conj(X') + i conj(Y') (mode -b); Z' and conj(Z')
            v.FA[(int64_t)b * nxn + i] = make_float2((Xr - Yi) * inv_n, (Xi + Yr) * inv_n);
            v.FB[(int64_t)b * nxn + i] = make_float2(zr * inv_n, zi * inv_n);
            if (bm != b) {
                v.FA[(int64_t)bm * nxn + i] = make_float2((Xr + Yi) * inv_n, (Yr - Xi) * inv_n);
                v.FB[(int64_t)bm * nxn + i] = make_float2(zr * inv_n, -zi * inv_n);
            }
        }
        __syncthreads();
    }
    grid.sync();
    transpose2(v.FA, v.FB, v.GA, v.GB, ny, nxn, sm);           // -> [column][mode]
    grid.sync();
    fft_rows(v.GA, v.GB, nxn, ny, v.ly, v.twy, true, sm);    // back along y
    grid.sync();
    for (int64_t e = tid; e < N; e += stride) {
        const int j = (int)(e / nxn), i = (int)(e - (int64_t)j * nxn);
        const float2 a = v.GA[(int64_t)i * ny + j], z = v.GB[(int64_t)i * ny + j];
        out[e] = V4<float>{a.x, a.y, z.x, 0.f};
    }
}

// RHS, initial guess (E^n), FP32 S / dA and FP32 block-Jacobi inverse.  A
// wall node (a box with walls) is vacuum: its x row has the one-sided curl_h of
// the inside cell column, its y and z rows are the time-centred Mur condition
// with right-hand side (E_w + E_v)/dt, at x = 0 for the field minus the
// incident wave (inc: the wave at the wall node and its neighbour at the old
// and new times), whose centred values move to the right-hand side.
template <typename R>
__global__ void k_cn_setup(GridArgs<double> g, const V4<R> *__restrict__ E, const V4<R> *__restrict__ H,
                           const double *__restrict__ M, CNVec v, double c2, WallRows wr, Inc inc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nxn || j >= g.ny) return;
    int64_t node = (int64_t)j * g.nxn + i;
    int im = (i == 0) ? g.nx - 1 : i - 1;
    int jm = (j == 0) ? g.ny - 1 : j - 1;
    if (!g.periodic_x && (i == 0 || i == g.nx)) {
        const int ic = (i == 0) ? 0 : g.nx - 1, iv = (i == 0) ? 1 : g.nx - 1;
        const V4<R> e = E[node], ev = E[(int64_t)j * g.nxn + iv];
        const V4<R> up = H[(int64_t)j * g.nx + ic], dn = H[(int64_t)jm * g.nx + ic];
        double ry = ((double)e.y + (double)ev.y) / g.dt, rz = ((double)e.z + (double)ev.z) / g.dt;
        if (i == 0) {
            ry += -(inc.old0[1] + inc.old1[1]) / g.dt + wr.cw * 0.5 * (inc.old0[1] + inc.new0[1]) +
                  wr.cv * 0.5 * (inc.old1[1] + inc.new1[1]);
            rz += -(inc.old0[2] + inc.old1[2]) / g.dt + wr.cw * 0.5 * (inc.old0[2] + inc.new0[2]) +
                  wr.cv * 0.5 * (inc.old1[2] + inc.new1[2]);
        }
        v.b[node] = V4<double>{(double)e.x + 0.5 * g.dt * (((double)up.z - (double)dn.z) * g.inv_dy), ry, rz, 0.0};
        v.x[node] = V4<double>{(double)e.x, (double)e.y, (double)e.z, 0.0};
        for (int k = 0; k < 9; ++k) {
            v.S[(int64_t)k * g.nnode + node] = 0.f;
            v.minv[(int64_t)k * g.nnode + node] = 0.f;
        }
        // diagonal of the wall rows: 1 + (dt/2)^2 / dy^2 (x), cw (y, z)
        v.minv[node] = (float)(1.0 / (1.0 + c2 * g.inv_dy * g.inv_dy));
        v.minv[4 * g.nnode + node] = (float)(1.0 / wr.cw);
        v.minv[8 * g.nnode + node] = (float)(1.0 / wr.cw);
        return;
    }
    V4<R> a = H[(int64_t)j * g.nx + i], b = H[(int64_t)j * g.nx + im];
    V4<R> c = H[(int64_t)jm * g.nx + i], d = H[(int64_t)jm * g.nx + im];
    double hy = 0.5 * g.inv_dy, hx = 0.5 * g.inv_dx;
    double cx = (((double)a.z + (double)b.z) - ((double)c.z + (double)d.z)) * hy;
    double cy = -((((double)a.z + (double)c.z) - ((double)b.z + (double)d.z)) * hx);
    double cz = (((double)a.y + (double)c.y) - ((double)b.y + (double)d.y)) * hx -
                (((double)a.x + (double)b.x) - ((double)c.x + (double)d.x)) * hy;
    double ia = g.inv_dx * g.inv_dy;
    V4<R> e = E[node];
    double hdt = 0.5 * g.dt;
    v.b[node] = V4<double>{(double)e.x + hdt * (cx - (double)M[10 * g.nnode + node] * ia),
                           (double)e.y + hdt * (cy - (double)M[11 * g.nnode + node] * ia),
                           (double)e.z + hdt * (cz - (double)M[12 * g.nnode + node] * ia), 0.0};
    v.x[node] = V4<double>{(double)e.x, (double)e.y, (double)e.z, 0.0};
    double A[9];
    for (int k = 0; k < 9; ++k) {
        A[k] = (double)M[(int64_t)(1 + k) * g.nnode + node] * ia;
        v.S[(int64_t)k * g.nnode + node] = (float)A[k];
    }
    // diagonal of (dt/2)^2 curl_h curl_e: (1/dy^2, 1/dx^2, 1/dx^2 + 1/dy^2)
    A[0] += 1.0 + c2 * g.inv_dy * g.inv_dy;
    A[4] += 1.0 + c2 * g.inv_dx * g.inv_dx;
    A[8] += 1.0 + c2 * (g.inv_dx * g.inv_dx + g.inv_dy * g.inv_dy);
    double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    double id = 1.0 / det;
    double inv[9] = {c00 * id, (A[2] * A[7] - A[1] * A[8]) * id, (A[1] * A[5] - A[2] * A[4]) * id,
                     c01 * id, (A[0] * A[8] - A[2] * A[6]) * id, (A[2] * A[3] - A[0] * A[5]) * id,
                     c02 * id, (A[1] * A[6] - A[0] * A[7]) * id, (A[0] * A[4] - A[1] * A[3]) * id};
    for (int k = 0; k < 9; ++k) v.minv[(int64_t)k * g.nnode + node] = (float)inv[k];
}

// Block sum of up to 3 values; thread 0 writes them to part[k * nb + block].
// The threads' values meet in shared memory and warp 0 adds them (strided
// lanes, then a butterfly), so that the FP64 adds run in one warp.
constexpr int CN_BS = 256;
__device__ inline void block_partials(double a0, double a1, double a2, int nv, double *part, int nb) {
    __shared__ double sh[3][CN_BS];
    const double v[3] = {a0, a1, a2};
    for (int k = 0; k < nv; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int k = 0; k < nv; ++k) {
            double s = sh[k][threadIdx.x];
            for (int j = threadIdx.x + 32; j < CN_BS; j += 32) s += sh[k][j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) part[(int64_t)k * nb + blockIdx.x] = s;
        }
    }
    __syncthreads();
}

// Fixed-order sum of the partials, identical in every block: lane l of warp 0
// adds partials l, l + 32, ..., then a butterfly over the lanes.  (One thread
// adding all nb partials kept the narrow FP64 pipe busy for nb instructions
// in every block.)  The partials come from other blocks: read through L2.
__device__ inline void reduce_partials(const double *part, int nb, int nv, double *out) {
    __shared__ double res[3];
    if (threadIdx.x < 32) {
        for (int k = 0; k < nv; ++k) {
            double s = 0.0;
            for (int b = threadIdx.x; b < nb; b += 32) s += __ldcg(part + (int64_t)k * nb + b);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (threadIdx.x == 0) res[k] = s;
        }
    }
    __syncthreads();
    for (int k = 0; k < nv; ++k) out[k] = res[k];
    __syncthreads();
}

// The whole solve in one cooperative launch (grid-wide barriers between the
// dependent phases).  Thread partial sums of the FP32 phases are FP32 (a few
// nodes per thread), block and grid sums FP64 in a fixed order.
// out = [FP32 iterations, relative FP64 residual, refinements].
__global__ void k_cn_solve(GridArgs<double> g, const double *__restrict__ Md, CNVec v, double c2, double tol,
                           int max_iter, double *part, double *out, WallRows wr) {
    cg::grid_group grid = cg::this_grid();
    const int64_t N = g.nnode;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int nb = gridDim.x;
    const double ia = g.inv_dx * g.inv_dy;
    const double hx = 0.5 * g.inv_dx, hy = 0.5 * g.inv_dy;
    const float c2f = (float)c2, hxf = (float)hx, hyf = (float)hy, cwf = (float)wr.cw, cvf = (float)wr.cv;
    double *pa = part, *pb = part + 3 * (int64_t)nb;  // alternating partial buffers
    int flip = 0;
    auto P = [&]() { double *q = flip ? pb : pa; flip ^= 1; return q; };
    const V4<float> zero4{0.f, 0.f, 0.f, 0.f};
    double red[3];
    double bnorm = -1.0, res = 0.0, rr_prev = 0.0;
    int total = 0, outer = 0;
    extern __shared__ float2 cn_sm[];
    float sx = 0.f, sy = 0.f, sz = 0.f;
    if (v.fft) {
        // twiddles, and the grid means of the diagonal of S for the preconditioner
        const int hxn = g.nx / 2, hyn = g.ny / 2;
        for (int64_t t = tid; t < hxn + hyn; t += stride) {
            double sn, cs;
            if (t < hxn) {
                sincospi(-2.0 * (double)t / g.nx, &sn, &cs);
                v.twx[t] = make_float2((float)cs, (float)sn);
            } else {
                sincospi(-2.0 * (double)(t - hxn) / g.ny, &sn, &cs);
                v.twy[t - hxn] = make_float2((float)cs, (float)sn);
            }
        }
        double a0 = 0, a1 = 0, a2 = 0;
        for (int64_t n = tid; n < N; n += stride) {
            a0 += v.S[n];
            a1 += v.S[4 * N + n];
            a2 += v.S[8 * N + n];
        }
        double *q0 = P();
        block_partials(a0, a1, a2, 3, q0, nb);
        grid.sync();
        reduce_partials(q0, nb, 3, red);
        sx = (float)(red[0] / N);
        sy = (float)(red[1] / N);
        sz = (float)(red[2] / N);
    } else if (v.line) {
        line_setup(grid, g, v, c2f, cwf, cvf);
        grid.sync();
    }
    for (;;) {
        // FP64 residual r = b - A x, handed to the FP32 solve; d = 0, r0 = r, p = v = 0
        double s_rr = 0, s_bb = 0;
        const int64_t NC = (int64_t)g.nx * g.ny;
        for (int64_t c = tid; c < NC; c += stride) {
            const int ci = (int)(c % g.nx), cj = (int)(c / g.nx);
            v.cc[c] = cell_curl_e(g, v.x, hx, hy, ci, cj);
        }
        grid.sync();
        for (int64_t n = tid; n < N; n += stride) {
            int i = (int)(n % g.nxn), j = (int)(n / g.nxn);
            V4<double> ax = apply_A_from_cells(g, v.x, v.cc, Md + N, ia, c2, hx, hy, i, j, wr.cw, wr.cv);
            V4<double> b = v.b[n];
            V4<double> r{b.x - ax.x, b.y - ax.y, b.z - ax.z, 0.0};
            V4<float> rf{(float)r.x, (float)r.y, (float)r.z, 0.f};
            v.r[n] = rf;
            v.r0[n] = rf;
            v.p[n] = zero4;
            v.v[n] = zero4;
            v.d[n] = zero4;
            s_rr += dot(r, r);
            if (bnorm < 0) s_bb += dot(b, b);
        }
        double *q = P();
        block_partials(s_rr, s_bb, 0.0, 2, q, nb);
        grid.sync();
        reduce_partials(q, nb, 2, red);
        if (bnorm < 0) bnorm = sqrt(red[1]);
        const double rr = red[0];
        if (bnorm == 0.0) {
            for (int64_t n = tid; n < N; n += stride) v.x[n] = V4<double>{0, 0, 0, 0};
            res = 0.0;
            break;
        }
        res = sqrt(rr) / bnorm;
        // converged, out of budget, or no longer improving (FP64 rounding floor)
        if (res <= tol || total >= max_iter || outer >= CN_MAX_OUTER || (outer > 0 && rr > 0.25 * rr_prev)) break;
        rr_prev = rr;
        ++outer;
        // FP32 BiCGSTAB (block-Jacobi, right preconditioned) on A d = r
        const double stop = (double)CN_INNER_RTOL * sqrt(rr);
        double rho = rr, rho_old = 1.0, alpha = 1.0, omega = 1.0;
        while (total < max_iter) {
            const float beta = (float)((rho / rho_old) * (alpha / omega));
            const float omf = (float)omega;
            for (int64_t n = tid; n < N; n += stride) {
                V4<float> r = v.r[n], p = v.p[n], vv = v.v[n];
                V4<float> pn{r.x + beta * (p.x - omf * vv.x), r.y + beta * (p.y - omf * vv.y),
                             r.z + beta * (p.z - omf * vv.z), 0.f};
                v.p[n] = pn;
                if (!v.fft && !v.line) v.ph[n] = apply_minv(v.minv, N, n, pn);
            }
            if (v.fft) {
                grid.sync();
                apply_spectral(grid, g, v, v.p, v.ph, c2f, sx, sy, sz, cn_sm);
            } else if (v.line) {
                grid.sync();
                apply_line(grid, g, v, v.p, v.ph, c2f, cwf, cvf, cn_sm);
            }
            grid.sync();
            float s_r0v = 0.f;
            for (int64_t n = tid; n < N; n += stride) {
                int i = (int)(n % g.nxn), j = (int)(n / g.nxn);
                V4<float> av = apply_A<float>(g, v.ph, v.S, 1.f, c2f, hxf, hyf, i, j, cwf, cvf);
                v.v[n] = av;
                s_r0v += dot(v.r0[n], av);
            }
            q = P();
            block_partials(s_r0v, 0, 0, 1, q, nb);
            grid.sync();
            reduce_partials(q, nb, 1, red);
            if (red[0] == 0.0) break;
            alpha = rho / red[0];
            const float af = (float)alpha;
            float s_ss = 0.f;
            for (int64_t n = tid; n < N; n += stride) {
                V4<float> r = v.r[n], vv = v.v[n];
                V4<float> s{r.x - af * vv.x, r.y - af * vv.y, r.z - af * vv.z, 0.f};
                v.s[n] = s;
                if (!v.fft && !v.line) v.sh[n] = apply_minv(v.minv, N, n, s);
                s_ss += dot(s, s);
            }
            q = P();
            block_partials(s_ss, 0, 0, 1, q, nb);
            grid.sync();
            reduce_partials(q, nb, 1, red);
            ++total;
            if (sqrt(red[0]) <= stop) {
                for (int64_t n = tid; n < N; n += stride) {
                    V4<float> d = v.d[n], ph = v.ph[n];
                    v.d[n] = V4<float>{d.x + af * ph.x, d.y + af * ph.y, d.z + af * ph.z, 0.f};
                }
                break;
            }
            if (v.fft) {
                apply_spectral(grid, g, v, v.s, v.sh, c2f, sx, sy, sz, cn_sm);
                grid.sync();
            } else if (v.line) {
                apply_line(grid, g, v, v.s, v.sh, c2f, cwf, cvf, cn_sm);
                grid.sync();
            }
            float s_ts = 0.f, s_tt = 0.f;
            for (int64_t n = tid; n < N; n += stride) {
                int i = (int)(n % g.nxn), j = (int)(n / g.nxn);
                V4<float> at = apply_A<float>(g, v.sh, v.S, 1.f, c2f, hxf, hyf, i, j, cwf, cvf);
                v.t[n] = at;
                V4<float> s = v.s[n];
                s_ts += dot(at, s);
                s_tt += dot(at, at);
            }
            q = P();
            block_partials(s_ts, s_tt, 0, 2, q, nb);
            grid.sync();
            reduce_partials(q, nb, 2, red);
            if (red[1] == 0.0) break;
            omega = red[0] / red[1];
            const float of = (float)omega;
            float s_r0r = 0.f, s_rr2 = 0.f;
            for (int64_t n = tid; n < N; n += stride) {
                V4<float> d = v.d[n], ph = v.ph[n], sh = v.sh[n], s = v.s[n], t = v.t[n];
                v.d[n] = V4<float>{d.x + af * ph.x + of * sh.x, d.y + af * ph.y + of * sh.y,
                                   d.z + af * ph.z + of * sh.z, 0.f};
                V4<float> r{s.x - of * t.x, s.y - of * t.y, s.z - of * t.z, 0.f};
                v.r[n] = r;
                s_r0r += dot(v.r0[n], r);
                s_rr2 += dot(r, r);
            }
            q = P();
            block_partials(s_r0r, s_rr2, 0, 2, q, nb);
            grid.sync();
            reduce_partials(q, nb, 2, red);
            rho_old = rho;
            rho = red[0];
            if (sqrt(red[1]) <= stop || rho == 0.0 || omega == 0.0) break;
        }
        // x += d in FP64
        for (int64_t n = tid; n < N; n += stride) {
            V4<double> x = v.x[n];
            V4<float> d = v.d[n];
            v.x[n] = V4<double>{x.x + (double)d.x, x.y + (double)d.y, x.z + (double)d.z, 0.0};
        }
        grid.sync();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = (double)total;
        out[1] = res;
        out[2] = (double)outer;
    }
}

// E^{n+1} = 2X - E^n, E^{n+1/2} = X (padded).
template <typename R>
__global__ void k_cn_finish(GridArgs<R> g, const V4<double> *__restrict__ X, const V4<R> *__restrict__ E,
                            V4<R> *__restrict__ Enew, V4<R> *__restrict__ Ehalf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (i >= g.nxn || j >= g.ny) return;
    int64_t node = (int64_t)j * g.nxn + i;
    V4<double> x = X[node];
    V4<R> e = E[node];
    Enew[node] = V4<R>{(R)(2.0 * x.x - (double)e.x), (R)(2.0 * x.y - (double)e.y), (R)(2.0 * x.z - (double)e.z), R(0)};
    Ehalf[pidx(g, i, j)] = V4<R>{(R)x.x, (R)x.y, (R)x.z, R(0)};
}

// The moments are FP64 for the solver; the FP32 form adds its sum and its
// compensation term in FP64 first.
__global__ void k_moments_to_double(const float *__restrict__ Mf, const float *__restrict__ Mlo,
                                    double *__restrict__ Md, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) Md[t] = (double)Mf[t] + (Mlo ? (double)Mlo[t] : 0.0);
}

// --------------------------------------------------------------------------- host side

static dim3 node_grid(const pic_t *h, int bs) { return dim3((h->nxn + bs - 1) / bs, h->ny); }
static dim3 cell_grid(const pic_t *h, int bs) { return dim3((h->nx + bs - 1) / bs, h->ny); }

template <typename R>
static int fill_ghosts_t(pic_t *h, void *F) {
    GridArgs<R> g = grid_args<R>(h);
    int64_t total = 2 * (int64_t)h->G * h->nxp + (int64_t)h->ny * (h->nxp - h->nxn);   // ring entries
    k_fill_ghosts<R><<<(unsigned)((total + 255) / 256), 256, 0, h->st>>>(g, h->nyp, (V4<R> *)F);
    count_launch(h);
    return check_launch("k_fill_ghosts");
}

int fill_ghosts(pic_t *h, void *padded) { return h->fp32 ? fill_ghosts_t<float>(h, padded) : fill_ghosts_t<double>(h, padded); }

template <typename R>
static int node_average_t(pic_t *h, int hsrc, int bdst) {
    GridArgs<R> g = grid_args<R>(h);
    k_node_average<R><<<node_grid(h, 128), 128, 0, h->st>>>(g, (const V4<R> *)h->H[hsrc], (V4<R> *)h->B[bdst]);
    count_launch(h);
    if (int rc = check_launch("k_node_average")) return rc;
    return fill_ghosts_t<R>(h, h->B[bdst]);
}

int node_average(pic_t *h, int hsrc, int bdst) {
    return h->fp32 ? node_average_t<float>(h, hsrc, bdst) : node_average_t<double>(h, hsrc, bdst);
}

double host_laser(double t, double a0, double omega, double tau, double t0);

// The incident plane wave (reading of the missing source equation) at the x = 0
// wall node and its neighbour, at the times of E^n and E^{n+1} of this step, in
// the polarised component (y or z).
static Inc incident(const pic_t *h) {
    const pic_config &c = h->cfg;
    double t_new = (double)(h->step + 1) * c.dt, t_old = t_new - c.dt;
    Inc inc;
    int pc = (c.laser_pol == 0) ? 1 : 2;
    for (int k = 0; k < 3; ++k) {
        bool on = (k == pc) && !h->periodic_x;
        inc.new0[k] = on ? host_laser(t_new, c.laser_a0, c.laser_omega, c.laser_tau, c.laser_t0) : 0.0;
        inc.old0[k] = on ? host_laser(t_old, c.laser_a0, c.laser_omega, c.laser_tau, c.laser_t0) : 0.0;
        inc.new1[k] = on ? host_laser(t_new - c.dx, c.laser_a0, c.laser_omega, c.laser_tau, c.laser_t0) : 0.0;
        inc.old1[k] = on ? host_laser(t_old - c.dx, c.laser_a0, c.laser_omega, c.laser_tau, c.laser_t0) : 0.0;
    }
    return inc;
}

template <typename R>
static int field_literal_t(pic_t *h) {
    GridArgs<R> g = grid_args<R>(h);
    int en = 1 - h->ecur, hn = 1 - h->hcur;
    // the exact deposit rewrites every moment from its fixed-point sums; the others deposit into the
    // moments this solve has read and zeroed
    TouchArgs<R> tm{h->touch_all ? nullptr : h->touched, h->tnx, h->tny, h->ntx, h->det ? nullptr : (R *)h->M,
                    h->det ? nullptr : (R *)h->Mlo};
    k_field_E_literal<R><<<node_grid(h, 128), 128, 0, h->st>>>(g, (const V4<R> *)h->E[h->ecur],
                                                                (const V4<R> *)h->H[h->hcur], (const R *)h->M,
                                                                (const R *)h->Mlo, (V4<R> *)h->E[en],
                                                                (V4<R> *)h->Ehalf, tm);
    count_launch(h);
    if (int rc = check_launch("k_field_E_literal")) return rc;
    h->moments_cleared = !h->det;
    int nl = 1;
    if (!h->periodic_x) {
        const pic_config &c = h->cfg;
        Inc inc = incident(h);
        R kap = (R)((c.dt - c.dx) / (c.dt + c.dx));
        k_field_walls<R><<<(h->ny + 127) / 128, 128, 0, h->st>>>(g, (const V4<R> *)h->E[h->ecur],
                                                                  (const V4<R> *)h->H[h->hcur], (V4<R> *)h->E[en],
                                                                  (V4<R> *)h->Ehalf, inc, kap);
        count_launch(h);
        ++nl;
        if (int rc = check_launch("k_field_walls")) return rc;
    }
    k_field_H<R, R><<<cell_grid(h, 128), 128, 0, h->st>>>(g, (const V4<R> *)h->E[en], (const V4<R> *)h->H[h->hcur],
                                                          (V4<R> *)h->H[hn], (R)(0.5 * h->cfg.dt / h->cfg.dx),
                                                          (R)(0.5 * h->cfg.dt / h->cfg.dy));
    count_launch(h);
    ++nl;
    if (int rc = check_launch("k_field_H")) return rc;
    return 0;
}

int field_literal(pic_t *h) { return h->fp32 ? field_literal_t<float>(h) : field_literal_t<double>(h); }

// The spectral preconditioner applies to periodic power-of-two grids, the
// line preconditioner to boxes with walls whose ny is a power of two.
static bool cn_spectral(const pic_t *h) {
    return h->cfg.cn_precond != PIC_CN_PRECOND_JACOBI && h->periodic_x && (h->nx & (h->nx - 1)) == 0 &&
           (h->ny & (h->ny - 1)) == 0 && h->nx >= 2 && h->ny >= 2 && h->nx <= 4096 && h->ny <= 4096;
}

static bool cn_line(const pic_t *h) {
    if (h->cfg.cn_precond == PIC_CN_PRECOND_JACOBI || h->periodic_x || (h->ny & (h->ny - 1)) != 0 || h->ny < 2 ||
        h->ny > 4096 || line_sweep_bytes(h->nxn) > 200 * 1024)   // a mode's sweep must fit in shared memory
        return false;
    // automatic: block-Jacobi (on the 1024 x 512 foil the line preconditioner cuts the iterations from
    // 6 to 3 at c dt/dx = 0.4 and from 19 to 6 at 2, but each application costs ~7 block-Jacobi ones)
    return h->cfg.cn_precond == PIC_CN_PRECOND_FFT;
}

// floats of the line preconditioner's arrays: column means, factors, sweep work
static size_t cn_line_floats(const pic_t *h) {
    return (size_t)h->nxn * (3 + 16 * (size_t)(h->ny / 2 + 1));
}

static CNVec cn_views(pic_t *h, double **Md) {
    char *base = (char *)h->cn;
    const size_t n = (size_t)h->nnode;
    CNVec v;
    v.x = (V4<double> *)base;
    v.b = v.x + n;
    v.cc = v.b + n;                  // cells: nx * ny = n (periodic x)
    V4<float> *f = (V4<float> *)(v.cc + n);
    V4<float> **slots[9] = {&v.d, &v.r, &v.r0, &v.p, &v.v, &v.s, &v.t, &v.ph, &v.sh};
    for (int k = 0; k < 9; ++k) *slots[k] = f + k * n;
    v.minv = (float *)(f + 9 * n);
    v.S = v.minv + 9 * n;
    *Md = (double *)(v.S + 9 * n);   // 312 n bytes from the base: 8-byte aligned
    v.FA = (float2 *)(*Md + (size_t)NMOM * n);
    v.FB = v.FA + n;
    v.GA = v.FB + n;
    v.GB = v.GA + n;
    v.twx = v.GB + n;
    v.twy = v.twx + h->nx / 2 + 1;
    auto log2i = [](int x) { int l = 0; while ((1 << l) < x) ++l; return l; };
    v.fft = cn_spectral(h) ? 1 : 0;
    v.lx = log2i(h->nx);
    v.ly = log2i(h->ny);
    v.line = cn_line(h) ? 1 : 0;
    v.scol = (float *)(v.twy + h->ny / 2 + 1);
    v.lf = v.scol + 3 * (size_t)h->nxn;
    v.lw = v.lf + 10 * (size_t)h->nxn * (h->ny / 2 + 1);
    return v;
}

// dynamic shared memory of the CN solve: two FFT row buffers and the
// per-stage twiddles (spectral preconditioner), else one transpose tile
static size_t cn_smem(const pic_t *h) {
    size_t nmax = (size_t)(h->nx > h->ny ? h->nx : h->ny);
    const size_t tile = 32 * 33 * sizeof(float2);
    if (cn_line(h)) nmax = (size_t)h->ny;   // its FFTs run along y only
    else if (!cn_spectral(h)) return tile;
    const size_t G = nmax > (size_t)FFT_GROUP ? nmax : (size_t)FFT_GROUP;
    size_t fft = (2 * G + nmax) * sizeof(float2);   // two row-group buffers and the per-stage twiddles
    if (cn_line(h) && line_sweep_bytes(h->nxn) > fft) fft = line_sweep_bytes(h->nxn);
    return fft > tile ? fft : tile;
}

size_t cn_bytes(const pic_t *h) {
    const size_t n = (size_t)h->nnode;
    return 3 * n * sizeof(V4<double>) + 9 * n * sizeof(V4<float>) + 18 * n * sizeof(float) +
           (size_t)NMOM * n * sizeof(double) + 4 * n * sizeof(float2) + (size_t)(h->nx + h->ny + 4) * sizeof(float2) +
           cn_line_floats(h) * sizeof(float) + 16;
}

template <typename R>
static int field_cn_t(pic_t *h) {
    GridArgs<R> g = grid_args<R>(h);
    GridArgs<double> gd = grid_args<double>(h);
    double *Md = nullptr;
    CNVec v = cn_views(h, &Md);
    const double *Msrc = (const double *)h->M;
    if (h->fp32) {
        int64_t n = (int64_t)NMOM * h->nnode;
        k_moments_to_double<<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>((const float *)h->M, (const float *)h->Mlo,
                                                                            Md, n);
        count_launch(h);
        if (int rc = check_launch("k_moments_to_double")) return rc;
        Msrc = Md;
    }
    double c2 = 0.25 * h->cfg.dt * h->cfg.dt;
    WallRows wr{1.0 / h->cfg.dt + 1.0 / h->cfg.dx, 1.0 / h->cfg.dt - 1.0 / h->cfg.dx};
    Inc inc = incident(h);
    k_cn_setup<R><<<node_grid(h, 128), 128, 0, h->st>>>(gd, (const V4<R> *)h->E[h->ecur], (const V4<R> *)h->H[h->hcur],
                                                         Msrc, v, c2, wr, inc);
    count_launch(h);
    if (int rc = check_launch("k_cn_setup")) return rc;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int bs = CN_BS;
    const size_t smem = cn_smem(h);
    // the whole grid must be resident: fix the shared-memory split before asking how many blocks fit
    cudaFuncSetAttribute(k_cn_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_cn_solve, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cn_solve, bs, smem);
    int nb = per_sm * nsm;
    int need = (int)((h->nnode + bs - 1) / bs);
    if (nb > need) nb = need;
    if (nb < 1) nb = 1;
    if (nb > h->cn_red_cap) {
        set_error("CN reduction scratch too small (%d < %d)", h->cn_red_cap, nb);
        return PIC_ERR_STATE;
    }
    double tol = h->cfg.cn_tol > 0 ? h->cfg.cn_tol : (h->fp32 ? 1e-10 : 1e-12);
    int maxit = h->cfg.cn_max_iter > 0 ? h->cfg.cn_max_iter : 400;
    void *args[] = {(void *)&gd, (void *)&Msrc, (void *)&v, (void *)&c2, (void *)&tol, (void *)&maxit,
                    (void *)&h->cn_red, (void *)&h->cn_out, (void *)&wr};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_cn_solve, dim3(nb), dim3(bs), args, smem, h->st);
    count_launch(h);
    if (e != cudaSuccess) {
        set_error("cudaLaunchCooperativeKernel(k_cn_solve): %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    int en = 1 - h->ecur, hn = 1 - h->hcur;
    k_cn_finish<R><<<node_grid(h, 128), 128, 0, h->st>>>(g, v.x, (const V4<R> *)h->E[h->ecur], (V4<R> *)h->E[en],
                                                          (V4<R> *)h->Ehalf);
    count_launch(h);
    if (int rc = check_launch("k_cn_finish")) return rc;
    k_field_H<R, double><<<cell_grid(h, 128), 128, 0, h->st>>>(g, v.x, (const V4<R> *)h->H[h->hcur], (V4<R> *)h->H[hn],
                                                               0.5 * h->cfg.dt / h->cfg.dx, 0.5 * h->cfg.dt / h->cfg.dy);
    count_launch(h);
    return check_launch("k_field_H(cn)");
}

int field_cn(pic_t *h) { return h->fp32 ? field_cn_t<float>(h) : field_cn_t<double>(h); }

// --------------------------------------------------------------------------- host <-> device field transfer

template <typename R>
__global__ void k_planar_to_v4(const double *__restrict__ src, int64_t n, V4<R> *__restrict__ dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = V4<R>{(R)src[t], (R)src[n + t], (R)src[2 * n + t], R(0)};
}

template <typename R>
__global__ void k_v4_to_planar(const V4<R> *__restrict__ src, int64_t n, double *__restrict__ dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        V4<R> v = src[t];
        dst[t] = (double)v.x;
        dst[n + t] = (double)v.y;
        dst[2 * n + t] = (double)v.z;
    }
}

template <typename R>
static int upload_fields_t(pic_t *h, const double *E3, const double *H3) {
    if (E3) {
        int64_t n = h->nnode;
        if (cudaMemcpyAsync(h->stage, E3, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return check_launch("upload E");
        k_planar_to_v4<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(h->stage, n, (V4<R> *)h->E[h->ecur]);
        count_launch(h);
        if (int rc = check_launch("k_planar_to_v4(E)")) return rc;
    }
    if (H3) {
        int64_t n = h->ncell;
        if (cudaMemcpyAsync(h->stage, H3, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return check_launch("upload H");
        k_planar_to_v4<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(h->stage, n, (V4<R> *)h->H[h->hcur]);
        count_launch(h);
        if (int rc = check_launch("k_planar_to_v4(H)")) return rc;
        cudaMemcpyAsync(h->H[1 - h->hcur], h->H[h->hcur], n * sizeof(V4<R>), cudaMemcpyDeviceToDevice, h->st);
    }
    return 0;
}

int upload_fields(pic_t *h, const double *E3, const double *H3) {
    return h->fp32 ? upload_fields_t<float>(h, E3, H3) : upload_fields_t<double>(h, E3, H3);
}

template <typename R>
static int download_fields_t(pic_t *h, double *E3, double *H3) {
    if (E3) {
        int64_t n = h->nnode;
        k_v4_to_planar<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>((const V4<R> *)h->E[h->ecur], n, h->stage);
        count_launch(h);
        if (int rc = check_launch("k_v4_to_planar(E)")) return rc;
        cudaMemcpyAsync(E3, h->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
        if (cudaStreamSynchronize(h->st) != cudaSuccess) return check_launch("download E");
    }
    if (H3) {
        int64_t n = h->ncell;
        k_v4_to_planar<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>((const V4<R> *)h->H[h->hcur], n, h->stage);
        count_launch(h);
        if (int rc = check_launch("k_v4_to_planar(H)")) return rc;
        cudaMemcpyAsync(H3, h->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
        if (cudaStreamSynchronize(h->st) != cudaSuccess) return check_launch("download H");
    }
    return 0;
}

int download_fields(pic_t *h, double *E3, double *H3) {
    return h->fp32 ? download_fields_t<float>(h, E3, H3) : download_fields_t<double>(h, E3, H3);
}

}  // namespace pic
