// FP64 global reductions of the state: kinetic energy sum w m (gamma - 1),
// particle charge sum q w, field energy 1/2 sum E^2 dA + 1/2 sum H^2 dA and the
// deposited charge sum rho dA.  Partials in FP64 are combined in a fixed tree
// (per block, per chunk of blocks, then over the chunks), so the result does
// not depend on scheduling; the sums, the particle counts, the removal
// counters, the sticky flags and the last CN solve's status come back to the
// host in one page-locked record.
//
// GB300 runs FP64 arithmetic at about 2 lanes per clock per SM, so the
// reductions keep FP64 work to whole warps that have something to add: empty
// tiles leave at once, a block's values meet in shared memory and one warp
// adds them, and the last step runs across the lanes of one warp.
#include "pic_internal.cuh"

namespace pic {

constexpr int DIAG_BLOCKS = 512;   // partials of the field sums
constexpr int DIAG_BS = 256;
constexpr int FINAL_BLOCKS = 32;   // chunks of the partials (one warp adds the chunks at the end)
constexpr int CHUNK_DOUBLES = 3 * PIC_MAX_SPECIES + 2;

// Block sum of v[0..NV) into thread 0's v (the other threads' v are left
// undefined): every thread stores its values, then warp 0 adds them in a
// fixed order (strided lanes, then a butterfly).
template <int NV>
__device__ inline void block_reduce(double (&v)[NV]) {
    __shared__ double red[NV][DIAG_BS];
    __syncthreads();   // a previous call's reads of red are done
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = red[k][threadIdx.x];
            for (int j = 1; j < DIAG_BS / 32; ++j) a += red[k][threadIdx.x + 32 * j];
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            v[k] = a;
        }
    }
}

// One block per tile bin, one warp per 32-slot segment (lane = slot):
// partial sums of w (gamma - 1), w and the particle count, into
// out[3 t + 0, 1, 2]; the species' m and q multiply them in k_diag_final.
// FP32 form: gamma - 1 = |u|^2 / (1 + gamma) in FP32 (no cancellation), the
// segment's 32 terms summed in FP32 by a fixed butterfly, the segment sums in
// FP64 by the warp's lane 0.  FP64 form: every term and sum in FP64, with
// gamma = (1 + |u|^2) / gamma from the carried 1/gamma of the particle's last
// deposit (made from the same u; no square root on the narrow FP64 pipe).
template <typename R>
__global__ void k_diag_bins(const int32_t *bstart, const int32_t *useg, const int32_t *segn, const R *ux, const R *uy,
                            const R *uz, const R *w, const double *__restrict__ ig, double *out) {
    const int u = useg[blockIdx.x];
    if (u == 0) {   // the whole block leaves
        if (threadIdx.x < 3) out[3 * blockIdx.x + threadIdx.x] = 0.0;
        return;
    }
    const int64_t sb = bstart[blockIdx.x] / SEG;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ke = 0, sw = 0;
    int cnt = 0;
    for (int j = wid; j < u; j += DIAG_BS / 32) {
        const int nseg = segn[sb + j];
        const bool valid = lane < nseg;
        if (lane == 0) cnt += nseg;
        const int64_t p = (sb + j) * SEG + lane;
        if (sizeof(R) == 4) {
            float kv = 0.f, wv = 0.f;
            if (valid) {
                const float a = (float)ux[p], b = (float)uy[p], c = (float)uz[p];
                const float uu = a * a + b * b + c * c;
                wv = (float)w[p];
                kv = wv * (uu / (1.f + sqrtf(1.f + uu)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kv += __shfl_xor_sync(0xffffffffu, kv, o);
                wv += __shfl_xor_sync(0xffffffffu, wv, o);
            }
            if (lane == 0) {
                ke += (double)kv;
                sw += (double)wv;
            }
        } else if (valid) {
            const double ww = w[p];
            const double a = ux[p], b = uy[p], c = uz[p];
            const double s = 1.0 + a * a + b * b + c * c;
            ke += ww * (ig ? fma(s, ig[p], -1.0) : sqrt(s) - 1.0);
            sw += ww;
        }
    }
    double v[3] = {ke, sw, (double)cnt};
    block_reduce<3>(v);
    if (threadIdx.x == 0) {
        out[3 * blockIdx.x] = v[0];
        out[3 * blockIdx.x + 1] = v[1];
        out[3 * blockIdx.x + 2] = v[2];
    }
}

// E energy with the node area (halved on walls), H energy (literal: H at the
// integer time as the mean of the two stored half-step values), and sum rho.
// The FP32 form squares and sums its few nodes per thread in FP32 (the FP64
// pipe is narrow); rho and every sum across threads are FP64.
template <typename R>
__global__ void k_diag_fields(GridArgs<double> g, const V4<R> *E, const V4<R> *H, const V4<R> *Hp, int avg,
                              const R *M, const R *Mlo, double *out) {
    R ee = 0, hh = 0;
    double rho = 0;
    const R area = (R)(g.dx * g.dy);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int step_i = (int)(stride % g.nxn);
    int i = (int)(t0 % g.nxn);   // column of node t, advanced with t
    for (int64_t t = t0; t < g.nnode; t += stride, i = (i + step_i >= g.nxn) ? i + step_i - g.nxn : i + step_i) {
        R a = area;
        if (!g.periodic_x && (i == 0 || i == g.nx)) a *= R(0.5);
        V4<R> e = E[t];
        ee += a * (e.x * e.x + e.y * e.y + e.z * e.z);
        rho += (double)M[t] + (Mlo ? (double)Mlo[t] : 0.0);
    }
    const int64_t nc = (int64_t)g.nx * g.ny;
    for (int64_t t = t0; t < nc; t += stride) {
        V4<R> v = H[t];
        R x = v.x, y = v.y, z = v.z;
        if (avg) {
            V4<R> u = Hp[t];
            x = R(0.5) * (x + u.x);
            y = R(0.5) * (y + u.y);
            z = R(0.5) * (z + u.z);
        }
        hh += area * (x * x + y * y + z * z);
    }
    double v[2] = {0.5 * ((double)ee + (double)hh), rho};
    block_reduce<2>(v);
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = v[0];
        out[2 * blockIdx.x + 1] = v[1];
    }
}

// Everything pic_diagnostics reports from the device, in one record.
struct DiagRecord {
    double kinetic, charge_particles, field, charge_grid, cn[3];
    int64_t count[PIC_MAX_SPECIES], removed[PIC_MAX_SPECIES];
    int32_t flags, pad;
};
constexpr int DIAG_RECORD_DOUBLES = (int)((sizeof(DiagRecord) + 7) / 8);

struct DiagSpecies {
    int live[PIC_MAX_SPECIES];   // the species has particle buffers (partials written)
    double q[PIC_MAX_SPECIES], m[PIC_MAX_SPECIES];
    int nsp;
};

// FINAL_BLOCKS blocks: block b sums its contiguous chunk of every species'
// tile partials and of the field partials into chunk[b]; the last block to
// finish (ticket) adds the chunks, lane c taking chunk c, in a fixed
// butterfly, and writes the record.  The ticket is zero at launch.
__global__ void k_diag_final(const double *part, int ntiles, DiagSpecies sp, const double *fpart, double *chunk,
                             unsigned *ticket, const int64_t *removed, const int32_t *flags, const double *cn_out,
                             DiagRecord *rec) {
    __shared__ bool last;
    const int b = blockIdx.x;
    double *mine = chunk + (size_t)b * CHUNK_DOUBLES;
    const int t0 = (int)((int64_t)ntiles * b / FINAL_BLOCKS), t1 = (int)((int64_t)ntiles * (b + 1) / FINAL_BLOCKS);
    for (int s = 0; s < sp.nsp; ++s) {
        double v[3] = {0, 0, 0};
        if (sp.live[s]) {
            const double *ps = part + (size_t)3 * ntiles * s;
            for (int i = t0 + threadIdx.x; i < t1; i += DIAG_BS) {
                v[0] += ps[3 * i];
                v[1] += ps[3 * i + 1];
                v[2] += ps[3 * i + 2];
            }
        }
        block_reduce<3>(v);
        if (threadIdx.x == 0)
            for (int k = 0; k < 3; ++k) mine[3 * s + k] = v[k];
    }
    {
        double v[2] = {0, 0};
        const int f0 = DIAG_BLOCKS * b / FINAL_BLOCKS, f1 = DIAG_BLOCKS * (b + 1) / FINAL_BLOCKS;
        for (int i = f0 + threadIdx.x; i < f1; i += DIAG_BS) {
            v[0] += fpart[2 * i];
            v[1] += fpart[2 * i + 1];
        }
        block_reduce<2>(v);
        if (threadIdx.x == 0) {
            mine[3 * PIC_MAX_SPECIES] = v[0];
            mine[3 * PIC_MAX_SPECIES + 1] = v[1];
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(ticket, 1u) == FINAL_BLOCKS - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    const int lane = threadIdx.x;
    static_assert(FINAL_BLOCKS == 32, "one lane per chunk");
    const double *c = chunk + (size_t)lane * CHUNK_DOUBLES;
    double ke = 0, qw = 0, cnt[PIC_MAX_SPECIES];
    for (int s = 0; s < sp.nsp; ++s) {
        double a = __ldcg(c + 3 * s), w = __ldcg(c + 3 * s + 1), n = __ldcg(c + 3 * s + 2);
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
            n += __shfl_xor_sync(0xffffffffu, n, o);
        }
        ke += sp.m[s] * a;
        qw += sp.q[s] * w;
        cnt[s] = n;
    }
    double fe = __ldcg(c + 3 * PIC_MAX_SPECIES), rho = __ldcg(c + 3 * PIC_MAX_SPECIES + 1);
    for (int o = 16; o > 0; o >>= 1) {
        fe += __shfl_xor_sync(0xffffffffu, fe, o);
        rho += __shfl_xor_sync(0xffffffffu, rho, o);
    }
    if (lane == 0) {
        rec->kinetic = ke;
        rec->charge_particles = qw;
        rec->field = fe;
        rec->charge_grid = rho;
        for (int k = 0; k < 3; ++k) rec->cn[k] = cn_out ? cn_out[k] : 0.0;
        for (int s = 0; s < PIC_MAX_SPECIES; ++s) {
            rec->count[s] = (s < sp.nsp) ? (int64_t)cnt[s] : 0;   // sums of integers below 2^53: exact
            rec->removed[s] = (s < sp.nsp) ? removed[s] : 0;
        }
        rec->flags = *flags;
        rec->pad = 0;
        *ticket = 0;
    }
}

template <typename R>
static int diag_t(pic_t *h, pic_diag *out) {
    const size_t np = 3 * (size_t)h->ntiles;   // partials per species
    double *fpart = h->d_diag + np * h->nsp;
    double *chunk = fpart + 2 * DIAG_BLOCKS;
    unsigned *ticket = (unsigned *)(chunk + (size_t)FINAL_BLOCKS * CHUNK_DOUBLES);
    DiagRecord *drec = (DiagRecord *)(chunk + (size_t)FINAL_BLOCKS * CHUNK_DOUBLES + 1);
    if ((size_t)h->diag_cap < np * h->nsp + 2 * DIAG_BLOCKS + (size_t)FINAL_BLOCKS * CHUNK_DOUBLES + 1 +
                                  DIAG_RECORD_DOUBLES) {
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
        sp.live[s] = 1;
        int b = S.bins;
        // the carried 1/gamma matches u once the moments are current (the caller has settled them)
        const double *ig = (!h->fp32 && !h->moments_stale) ? S.carry[b] : nullptr;
        k_diag_bins<R><<<h->ntiles, DIAG_BS, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], (const R *)S.ux[b],
                                                        (const R *)S.uy[b], (const R *)S.uz[b], (const R *)S.w[b], ig,
                                                        h->d_diag + np * s);
        count_launch(h);
        if (int rc = check_launch("k_diag_bins")) return rc;
    }
    int avg = (h->cfg.field_mode == PIC_FIELD_LITERAL) ? 1 : 0;
    k_diag_fields<R><<<DIAG_BLOCKS, DIAG_BS, 0, h->st>>>(grid_args<double>(h), (const V4<R> *)h->E[h->ecur],
                                                        (const V4<R> *)h->H[h->hcur], (const V4<R> *)h->H[1 - h->hcur],
                                                        avg, (const R *)h->M, (const R *)h->Mlo, fpart);
    count_launch(h);
    if (int rc = check_launch("k_diag_fields")) return rc;
    cudaMemsetAsync(ticket, 0, sizeof(unsigned), h->st);
    k_diag_final<<<FINAL_BLOCKS, DIAG_BS, 0, h->st>>>(h->d_diag, h->ntiles, sp, fpart, chunk, ticket, h->d_removed,
                                                      h->d_flags, h->cn_out, drec);
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

// Raw node sums (+ the FP32 compensation) per unit area: times 1/(dx dy),
// twice that on a wall column (half a cell's area) -- the moments reported
// for the next solve.
template <typename R>
__global__ void k_moments_out(const R *__restrict__ M, const R *__restrict__ Mlo, int64_t nnode, int nxn, int nx,
                              int walls, double inv_area, double *__restrict__ out) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nnode; n += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(n % nxn);
        const double f = (walls && (i == 0 || i == nx)) ? 2.0 * inv_area : inv_area;   // wall nodes: half a cell
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            const int64_t t = (int64_t)k * nnode + n;
            const double v = Mlo ? (double)M[t] + (double)Mlo[t] : (double)M[t];
            out[t] = v * f;
        }
    }
}

int moments_to_stage(pic_t *h) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (h->nnode + 255) / 256;
    if (blocks > 8 * (int64_t)nsm) blocks = 8 * (int64_t)nsm;
    if (blocks < 1) blocks = 1;
    const double inv_area = 1.0 / (h->cfg.dx * h->cfg.dy);
    if (h->fp32)
        k_moments_out<float><<<(unsigned)blocks, 256, 0, h->st>>>((const float *)h->M, (const float *)h->Mlo, h->nnode,
                                                                 h->nxn, h->nx, h->periodic_x ? 0 : 1, inv_area,
                                                                 h->stage);
    else
        k_moments_out<double><<<(unsigned)blocks, 256, 0, h->st>>>((const double *)h->M, nullptr, h->nnode, h->nxn,
                                                                  h->nx, h->periodic_x ? 0 : 1, inv_area, h->stage);
    count_launch(h);
    return check_launch("k_moments_out");
}

// tile partials, field partials, chunk partials, the ticket, the record
int diag_scratch_doubles(int nsp, int ntiles) {
    return 3 * ntiles * nsp + 2 * DIAG_BLOCKS + FINAL_BLOCKS * CHUNK_DOUBLES + 1 + DIAG_RECORD_DOUBLES;
}

size_t diag_record_bytes() { return sizeof(DiagRecord); }

}  // namespace pic

// --------------------------------------------------------------------------- FP64 rate probe

namespace pic {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_ITERS = 4096;   // x 4 unrolled steps of 8 FMAs per thread

// Independent FMA chains a <- a b + c (|b| < 1 keeps the values bounded); the
// results are stored so that no chain can be removed.
__global__ void __launch_bounds__(256) k_fp64_rate(double *__restrict__ out, double b, double c) {
    double a[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = 1e-3 * (threadIdx.x + 1) + k;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace pic

extern "C" PIC_API int pic_probe_fp64_rate(void *cuda_stream, int repeats, double *tflops) {
    using namespace pic;
    if (!tflops || repeats < 1) {
        set_error("pic_probe_fp64_rate: NULL result or repeats < 1");
        return PIC_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 8 * (nsm > 0 ? nsm : 1), threads = 256;
    double *d = nullptr;
    if (cudaMalloc(&d, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("pic_probe_fp64_rate: allocation failed");
        return PIC_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    int rc = PIC_OK;
    for (int r = 0; r <= repeats && rc == PIC_OK; ++r) {
        cudaEventRecord(e0, st);
        k_fp64_rate<<<blocks, threads, 0, st>>>(d, 0.999999, 1e-7);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = check_launch("k_fp64_rate");
            if (!rc) rc = PIC_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * PROBE_CHAINS * 4.0 * PROBE_ITERS * (double)blocks * threads;
        if (r > 0 && ms > 0.f) {
            const double tf = flops / (ms * 1e-3) / 1e12;
            if (tf > best) best = tf;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    *tflops = best;
    return rc;
}
