// FP64 global reductions of the state: kinetic energy sum w m (gamma - 1),
// particle charge sum q w, field energy 1/2 sum E^2 dA + 1/2 sum H^2 dA and the
// deposited charge sum rho dA.  Per-block partials in FP64 are summed by one
// block in a fixed order, so the result does not depend on scheduling; the
// sums, the particle counts, the removal counters, the sticky flags and the
// last CN solve's status come back to the host in one page-locked record.
#include "pic_internal.cuh"

namespace pic {

constexpr int DIAG_BLOCKS = 512;
constexpr int DIAG_BS = 256;

// Block sum of (a, b) into out[2 blockIdx.x], out[2 blockIdx.x + 1].
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

// One block per tile bin, one warp per 32-slot segment (lane = slot):
// partial sums of w (gamma - 1) and w; the species' m and q multiply them in
// k_diag_final.
template <typename R>
__global__ void k_diag_bins(const int32_t *bstart, const int32_t *useg, const int32_t *segn, const R *ux, const R *uy,
                            const R *uz, const R *w, double *out) {
    const int64_t sb = bstart[blockIdx.x] / SEG;
    const int u = useg[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ke = 0, sw = 0;
    for (int j = wid; j < u; j += DIAG_BS / 32) {
        if (lane >= segn[sb + j]) continue;
        const int64_t p = (sb + j) * SEG + lane;
        const double ww = w[p];
        if (sizeof(R) == 4) {
            // FP32 form: gamma - 1 = |u|^2 / (1 + gamma) in FP32 (no cancellation), summed in FP64
            const float a = (float)ux[p], b = (float)uy[p], c = (float)uz[p];
            const float uu = a * a + b * b + c * c;
            ke += ww * (double)(uu / (1.f + sqrtf(1.f + uu)));
        } else {
            const double a = ux[p], b = uy[p], c = uz[p];
            ke += ww * (sqrt(1.0 + a * a + b * b + c * c) - 1.0);
        }
        sw += ww;
    }
    block_sum2(ke, sw, out);
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

// Everything pic_diagnostics reports from the device, in one record.
struct DiagRecord {
    double kinetic, charge_particles, field, charge_grid, cn[3];
    int64_t count[PIC_MAX_SPECIES], removed[PIC_MAX_SPECIES];
    int32_t flags, pad;
};
constexpr int DIAG_RECORD_DOUBLES = (int)((sizeof(DiagRecord) + 7) / 8);

struct DiagSpecies {
    const int32_t *count[PIC_MAX_SPECIES];   // &cstart[ntiles]; null for a species never loaded
    double q[PIC_MAX_SPECIES], m[PIC_MAX_SPECIES];
    int nsp;
};

// Thread 0 gets the block sums of (a, b); every thread may call it again.
__device__ inline void block_sum2_to0(double &a, double &b) {
    __shared__ double s[2][DIAG_BS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();   // the previous call's reads of s are done
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) { s[0][wid] = a; s[1][wid] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0;
        b = 0;
        for (int w = 0; w < DIAG_BS / 32; ++w) { a += s[0][w]; b += s[1][w]; }
    }
}

// One block: per species, the tile partials (in tile order per thread, then a
// fixed tree) times m and q; the field partials; the counters.
__global__ void k_diag_final(const double *part, int np, DiagSpecies sp, const double *fpart, const int64_t *removed,
                             const int32_t *flags, const double *cn_out, DiagRecord *rec) {
    double ke = 0, qw = 0;
    for (int s = 0; s < sp.nsp; ++s) {
        double a = 0, b = 0;
        if (sp.count[s])
            for (int i = threadIdx.x; i < np / 2; i += DIAG_BS) {
                a += part[(size_t)np * s + 2 * i];
                b += part[(size_t)np * s + 2 * i + 1];
            }
        block_sum2_to0(a, b);
        if (threadIdx.x == 0) {
            ke += sp.m[s] * a;
            qw += sp.q[s] * b;
        }
    }
    double fe = 0, rho = 0;
    for (int i = threadIdx.x; i < DIAG_BLOCKS; i += DIAG_BS) {
        fe += fpart[2 * i];
        rho += fpart[2 * i + 1];
    }
    block_sum2_to0(fe, rho);
    if (threadIdx.x == 0) {
        rec->kinetic = ke;
        rec->charge_particles = qw;
        rec->field = fe;
        rec->charge_grid = rho;
        for (int k = 0; k < 3; ++k) rec->cn[k] = cn_out ? cn_out[k] : 0.0;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            rec->count[s] = (s < sp.nsp && sp.count[s]) ? (int64_t)*sp.count[s] : 0;
            rec->removed[s] = (s < sp.nsp) ? removed[s] : 0;
        }
        rec->flags = *flags;
        rec->pad = 0;
    }
}

template <typename R>
static int diag_t(pic_t *h, pic_diag *out) {
    const int np = 2 * h->ntiles;  // partials per species
    const int need = np * h->nsp + 2 * DIAG_BLOCKS;
    if (h->diag_cap < need + DIAG_RECORD_DOUBLES) {
        set_error("diagnostics scratch too small");
        return PIC_ERR_STATE;
    }
    DiagSpecies sp = {};
    sp.nsp = h->nsp;
    for (int s = 0; s < h->nsp; ++s) {
        SpeciesBuf &S = h->sp[s];
        sp.q[s] = S.q;
        sp.m[s] = S.m;
        if (S.cap == 0) continue;
        // live count per tile and its prefix (device only; read back in the record)
        if (int rc = tile_counts(h, s)) return rc;
        if (int rc = scan_tiles(h, S.tcount, S.cstart)) return rc;
        sp.count[s] = S.cstart + h->ntiles;
        int b = S.bins;
        k_diag_bins<R><<<h->ntiles, DIAG_BS, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], (const R *)S.ux[b],
                                                        (const R *)S.uy[b], (const R *)S.uz[b], (const R *)S.w[b],
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
    DiagRecord *drec = (DiagRecord *)(h->d_diag + need);
    k_diag_final<<<1, DIAG_BS, 0, h->st>>>(h->d_diag, np, sp, fpart, h->d_removed, h->d_flags, h->cn_out, drec);
    count_launch(h);
    if (int rc = check_launch("k_diag_final")) return rc;
    DiagRecord *rec = (DiagRecord *)h->h_diag;
    cudaError_t e = cudaMemcpyAsync(rec, drec, sizeof(DiagRecord), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        set_error("diagnostics readback: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    out->kinetic = rec->kinetic;
    out->charge_particles = rec->charge_particles;
    out->field = rec->field;
    out->total = rec->kinetic + rec->field;
    out->charge_grid = rec->charge_grid;
    out->count = 0;
    out->removed = 0;
    for (int s = 0; s < h->nsp; ++s) {
        if (h->sp[s].cap) {
            h->sp[s].n = rec->count[s];
            h->sp[s].n_exact = true;
        }
        out->count += h->sp[s].n;
        out->removed += rec->removed[s];
    }
    out->cn_iterations = (int32_t)rec->cn[0];
    out->cn_residual = rec->cn[1];
    out->cn_refinements = (int32_t)rec->cn[2];
    out->flags = rec->flags;
    return 0;
}

int diagnostics(pic_t *h, pic_diag *out) { return h->fp32 ? diag_t<float>(h, out) : diag_t<double>(h, out); }

int diag_scratch_doubles(int nsp, int ntiles) { return 2 * ntiles * nsp + 2 * DIAG_BLOCKS + DIAG_RECORD_DOUBLES; }

size_t diag_record_bytes() { return sizeof(DiagRecord); }

}  // namespace pic
