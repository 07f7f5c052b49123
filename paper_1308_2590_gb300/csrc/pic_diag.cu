// FP64 global reductions of the state: kinetic energy sum w m (gamma - 1),
// particle charge sum q w, field energy 1/2 sum E^2 dA + 1/2 sum H^2 dA and the
// deposited charge sum rho dA.  Per-block partials in FP64 are summed on the
// host in block order, so the result does not depend on scheduling.
#include "pic_internal.cuh"

namespace pic {

constexpr int DIAG_BLOCKS = 512;
constexpr int DIAG_BS = 256;

__device__ inline void block_sum2(double a, double b, double *out) {
    __shared__ double s[2][DIAG_BS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { s[0][wid] = a; s[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int w = 0; w < DIAG_BS / 32; ++w) { x += s[0][w]; y += s[1][w]; }
        out[2 * blockIdx.x] = x;
        out[2 * blockIdx.x + 1] = y;
    }
}

// One block per tile bin.
template <typename R>
__global__ void k_diag_bins(const int32_t *bstart, const int32_t *useg, const int32_t *segn, const R *ux, const R *uy,
                            const R *uz, const R *w, double q, double m, double *out) {
    const int64_t b0 = bstart[blockIdx.x];
    const int u = useg[blockIdx.x];
    double ke = 0, qw = 0;
    for (int64_t i = threadIdx.x; i < (int64_t)u * SEG; i += blockDim.x) {
        const int64_t j = i / SEG;
        if ((int)(i - j * SEG) >= segn[b0 / SEG + j]) continue;
        const int64_t p = b0 + i;
        const double ww = w[p];
        if (sizeof(R) == 4) {
            // FP32 form: gamma - 1 = |u|^2 / (1 + gamma) in FP32 (no cancellation), summed in FP64
            const float a = (float)ux[p], b = (float)uy[p], c = (float)uz[p];
            const float uu = a * a + b * b + c * c;
            ke += ww * m * (double)(uu / (1.f + sqrtf(1.f + uu)));
        } else {
            const double a = ux[p], b = uy[p], c = uz[p];
            ke += ww * m * (sqrt(1.0 + a * a + b * b + c * c) - 1.0);
        }
        qw += q * ww;
    }
    block_sum2(ke, qw, out);
}

// E energy with the node area (halved on walls), H energy (literal: H at the
// integer time as the mean of the two stored half-step values), and sum rho.
template <typename R>
__global__ void k_diag_fields(GridArgs<double> g, const V4<R> *E, const V4<R> *H, const V4<R> *Hp, int avg,
                              const R *M, const R *Mlo, double *out) {
    double ee = 0, hh = 0, rho = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.nnode; t += stride) {
        int i = (int)(t % g.nxn);
        double a = g.dx * g.dy;
        if (!g.periodic_x && (i == 0 || i == g.nx)) a *= 0.5;
        V4<R> e = E[t];
        ee += a * ((double)e.x * e.x + (double)e.y * e.y + (double)e.z * e.z);
        rho += (double)M[t] + (Mlo ? (double)Mlo[t] : 0.0);
    }
    int64_t nc = (int64_t)g.nx * g.ny;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += stride) {
        V4<R> v = H[t];
        double x = v.x, y = v.y, z = v.z;
        if (avg) {
            V4<R> u = Hp[t];
            x = 0.5 * (x + (double)u.x);
            y = 0.5 * (y + (double)u.y);
            z = 0.5 * (z + (double)u.z);
        }
        hh += g.dx * g.dy * (x * x + y * y + z * z);
    }
    block_sum2(0.5 * (ee + hh), rho, out);
}

template <typename R>
static int diag_t(pic_t *h, pic_diag *out) {
    const int np = 2 * h->ntiles;  // partials per species
    int need = np * h->nsp + 2 * DIAG_BLOCKS;
    if (h->diag_cap < need) {
        set_error("diagnostics scratch too small");
        return PIC_ERR_STATE;
    }
    for (int s = 0; s < h->nsp; ++s) {
        SpeciesBuf &S = h->sp[s];
        if (S.cap == 0) {
            cudaMemsetAsync(h->d_diag + (size_t)np * s, 0, np * sizeof(double), h->st);
            continue;
        }
        int b = S.bins;
        k_diag_bins<R><<<h->ntiles, DIAG_BS, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], (const R *)S.ux[b],
                                                        (const R *)S.uy[b],
                                                        (const R *)S.uz[b], (const R *)S.w[b], S.q, S.m,
                                                        h->d_diag + (size_t)np * s);
        count_launch(h);
        if (int rc = check_launch("k_diag_bins")) return rc;
    }
    int avg = (h->cfg.field_mode == PIC_FIELD_LITERAL) ? 1 : 0;
    double *fpart = h->d_diag + (size_t)np * h->nsp;
    k_diag_fields<R><<<DIAG_BLOCKS, DIAG_BS, 0, h->st>>>(grid_args<double>(h), (const V4<R> *)h->E[h->ecur],
                                                        (const V4<R> *)h->H[h->hcur], (const V4<R> *)h->H[1 - h->hcur],
                                                        avg, (const R *)h->M, (const R *)h->Mlo, fpart);
    count_launch(h);
    if (int rc = check_launch("k_diag_fields")) return rc;
    double *host = new double[need];
    cudaError_t e = cudaMemcpyAsync(host, h->d_diag, need * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        delete[] host;
        set_error("diagnostics readback: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    double ke = 0, qw = 0;
    for (int s = 0; s < h->nsp; ++s)
        for (int b = 0; b < h->ntiles; ++b) {
            ke += host[(size_t)np * s + 2 * b];
            qw += host[(size_t)np * s + 2 * b + 1];
        }
    double fe = 0, rho = 0;
    for (int b = 0; b < DIAG_BLOCKS; ++b) {
        fe += host[(size_t)np * h->nsp + 2 * b];
        rho += host[(size_t)np * h->nsp + 2 * b + 1];
    }
    delete[] host;
    out->kinetic = ke;
    out->charge_particles = qw;
    out->field = fe;
    out->total = ke + fe;
    out->charge_grid = rho;
    return 0;
}

int diagnostics(pic_t *h, pic_diag *out) { return h->fp32 ? diag_t<float>(h, out) : diag_t<double>(h, out); }

int diag_scratch_doubles(int nsp, int ntiles) { return 2 * ntiles * nsp + 2 * DIAG_BLOCKS; }

}  // namespace pic
