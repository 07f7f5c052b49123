// C ABI of libpic (include/pic.h): handle life cycle, device memory, the
// order of one PIC cycle (Section 3.3: field solver, forces, pusher,
// moments), host <-> device transfers and error reporting.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "pic_internal.cuh"

namespace pic {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}

double host_laser(double t, double a0, double omega, double tau, double t0) {
    if (t < 0.0 || a0 == 0.0) return 0.0;
    double env = (tau > 0.0) ? exp(-2.0 * log(2.0) * (t - t0) * (t - t0) / (tau * tau)) : 1.0;
    return a0 * sin(omega * t) * env;
}

size_t cn_bytes(const pic_t *h);
int diag_scratch_doubles(int nsp, int ntiles);
size_t diag_record_bytes();
void tile_free(pic_t *h);

// --------------------------------------------------------------------------- event-based timing (no host sync)

struct PendingEv {
    int cls;
    int nlaunch;
    cudaEvent_t a, b;
};
struct TimingState {
    std::vector<PendingEv> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t open = nullptr;
};
static TimingState &tstate(pic_t *h);

}  // namespace pic

struct pic_timing_holder {
    pic::TimingState st;
};

namespace pic {

static cudaEvent_t take_event(TimingState &t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace pic

// The timing state lives beside the handle (allocated on first use).
static std::vector<std::pair<pic_t *, pic_timing_holder *>> g_timing_states;
static std::mutex g_timing_mu;   // handles may live in several threads (the server's worker, the caller)

namespace pic {

static TimingState &tstate(pic_t *h) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (auto &p : g_timing_states)
        if (p.first == h) return p.second->st;
    g_timing_states.push_back({h, new pic_timing_holder()});
    return g_timing_states.back().second->st;
}

static void tstate_free(pic_t *h) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    for (size_t k = 0; k < g_timing_states.size(); ++k)
        if (g_timing_states[k].first == h) {
            TimingState &t = g_timing_states[k].second->st;
            for (auto &p : t.pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
            for (auto e : t.pool) cudaEventDestroy(e);
            if (t.open) cudaEventDestroy(t.open);
            delete g_timing_states[k].second;
            g_timing_states.erase(g_timing_states.begin() + k);
            return;
        }
}

void timing_begin(pic_t *h) {
    if (!h->timing.enabled) return;
    TimingState &t = tstate(h);
    t.open = take_event(t);
    cudaEventRecord(t.open, h->st);
}

void timing_end(pic_t *h, int cls, int nlaunch) {
    h->timing.launches[cls] += nlaunch;
    if (!h->timing.enabled) return;
    TimingState &t = tstate(h);
    cudaEvent_t b = take_event(t);
    cudaEventRecord(b, h->st);
    t.pending.push_back({cls, nlaunch, t.open, b});
    t.open = nullptr;
}

static int harvest(pic_t *h) {
    TimingState &t = tstate(h);
    if (t.pending.empty()) return 0;
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return check_launch("timing sync");
    for (auto &p : t.pending) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        h->timing.ms[p.cls] += ms;
        t.pool.push_back(p.a);
        t.pool.push_back(p.b);
    }
    t.pending.clear();
    return 0;
}

// --------------------------------------------------------------------------- memory helpers

static int dalloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) return 0;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes for %s failed", bytes, what);
        *p = nullptr;
        return PIC_ERR_OOM;
    }
    return 0;
}

int ensure_stage_doubles(pic_t *h, int64_t ndoubles) {
    if (ndoubles <= h->stage_cap) return 0;
    cudaStreamSynchronize(h->st);
    cudaFree(h->stage);
    h->stage = nullptr;
    int64_t cap = ndoubles + ndoubles / 4 + 1024;
    if (int rc = dalloc((void **)&h->stage, cap * sizeof(double), "staging")) return rc;
    h->stage_cap = cap;
    return 0;
}

static int ensure_stage(pic_t *h, int64_t ndoubles) { return ensure_stage_doubles(h, ndoubles); }

// Staging a handle starts with: field uploads and downloads (3 planes) and the
// 13 normalised moment planes of pic_moments.
static int64_t init_stage_doubles(const pic_t *h) {
    const int64_t f = 3 * (h->nnode > h->ncell ? h->nnode : h->ncell), m = (int64_t)NMOM * h->nnode;
    return f > m ? f : m;
}

static void free_particle_buffers(SpeciesBuf &S) {
    for (int b = 0; b < 3; ++b) {
        cudaFree(S.cell[b]); cudaFree(S.ox[b]); cudaFree(S.oy[b]);
        cudaFree(S.ux[b]); cudaFree(S.uy[b]); cudaFree(S.uz[b]); cudaFree(S.w[b]); cudaFree(S.carry[b]);
        S.cell[b] = nullptr; S.ox[b] = S.oy[b] = S.ux[b] = S.uy[b] = S.uz[b] = S.w[b] = nullptr;
        S.carry[b] = nullptr;
    }
    cudaFree(S.mkey);
    cudaFree(S.segn[0]);
    cudaFree(S.segn[1]);
    cudaFree(S.segml);
    S.mkey = nullptr;
    S.segn[0] = S.segn[1] = S.segml = nullptr;
    S.cap = 0;
}

static void free_species(SpeciesBuf &S) {
    free_particle_buffers(S);
    cudaFree(S.bstart); cudaFree(S.useg[0]); cudaFree(S.useg[1]); cudaFree(S.tcount); cudaFree(S.cstart);
    cudaFree(S.cend);
    S.bstart = S.useg[0] = S.useg[1] = S.tcount = S.cstart = S.cend = nullptr;
}

// Grow a species' three buffer sets to at least `slots` slots, keeping the
// current bins (their slot offsets stay valid).
static int ensure_species_capacity(pic_t *h, int s, int64_t slots) {
    SpeciesBuf &S = h->sp[s];
    if (slots <= S.cap) return 0;
    if (slots > (1ll << 30)) {
        set_error("species %d would need %lld particle slots (limit 2^30)", s, (long long)slots);
        return PIC_ERR_CAPACITY;
    }
    int64_t cap = slots;
    SpeciesBuf N;
    size_t rb = h->rs * cap;
    int rc = 0;
    for (int b = 0; b < 3 && !rc; ++b) {
        rc = dalloc((void **)&N.cell[b], cap * sizeof(int32_t), "particles");
        if (!rc) rc = dalloc(&N.ox[b], rb, "particles");
        if (!rc) rc = dalloc(&N.oy[b], rb, "particles");
        if (!rc) rc = dalloc(&N.ux[b], rb, "particles");
        if (!rc) rc = dalloc(&N.uy[b], rb, "particles");
        if (!rc) rc = dalloc(&N.uz[b], rb, "particles");
        if (!rc) rc = dalloc(&N.w[b], rb, "particles");
        if (!rc && !h->fp32) rc = dalloc((void **)&N.carry[b], (size_t)NCARRY * cap * sizeof(double), "particles");
    }
    if (!rc) rc = dalloc((void **)&N.mkey, cap * sizeof(uint32_t), "mirror keys");
    if (!rc) rc = dalloc((void **)&N.segn[0], (cap / SEG) * sizeof(int32_t), "segment counts");
    if (!rc) rc = dalloc((void **)&N.segn[1], (cap / SEG) * sizeof(int32_t), "segment counts");
    if (!rc) rc = dalloc((void **)&N.segml, (cap / SEG) * sizeof(int32_t), "segment counts");
    if (rc) {
        free_particle_buffers(N);
        return rc;
    }
    if (S.cap > 0) {
        int c = S.bins;
        int64_t keep = S.cap;
        cudaMemcpyAsync(N.cell[0], S.cell[c], keep * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->st);
        void *src[6] = {S.ox[c], S.oy[c], S.ux[c], S.uy[c], S.uz[c], S.w[c]};
        void *dst[6] = {N.ox[0], N.oy[0], N.ux[0], N.uy[0], N.uz[0], N.w[0]};
        for (int k = 0; k < 6; ++k) cudaMemcpyAsync(dst[k], src[k], keep * h->rs, cudaMemcpyDeviceToDevice, h->st);
        if (S.carry[c])
            for (int k = 0; k < NCARRY; ++k)
                cudaMemcpyAsync(N.carry[0] + k * cap, S.carry[c] + k * keep, keep * sizeof(double),
                                cudaMemcpyDeviceToDevice, h->st);
        cudaMemcpyAsync(N.segn[S.scur], S.segn[S.scur], (keep / SEG) * sizeof(int32_t), cudaMemcpyDeviceToDevice, h->st);
        cudaStreamSynchronize(h->st);
    }
    free_particle_buffers(S);
    for (int b = 0; b < 3; ++b) {
        S.cell[b] = N.cell[b]; S.ox[b] = N.ox[b]; S.oy[b] = N.oy[b];
        S.ux[b] = N.ux[b]; S.uy[b] = N.uy[b]; S.uz[b] = N.uz[b]; S.w[b] = N.w[b];
        S.carry[b] = N.carry[b];
    }
    S.mkey = N.mkey;
    S.segn[0] = N.segn[0];
    S.segn[1] = N.segn[1];
    S.segml = N.segml;
    S.bins = 0; S.mir = 1; S.spare = 2;
    S.cap = cap;
    return ensure_sort_capacity(h, 2 * cap);
}

// Sticky device flags -> error codes.
static int flag_error(int32_t f) {
    if (f & 4) {
        set_error("particle bins exceeded the allocated capacity");
        return PIC_ERR_CAPACITY;
    }
    if (f & 8) {
        set_error("a tile's TMA copy did not complete within the wait limit");
        return PIC_ERR_TIMEOUT;
    }
    if (f & 16) {
        set_error("a particle was found outside its bin's tile");
        return PIC_ERR_STATE;
    }
    if (f & FLAG_CHECK) {
        set_error("an invariant check of the checks build failed (index, offset, destination or canary)");
        return PIC_ERR_STATE;
    }
    return 0;
}

// A step's per-tile regroup is taken as the new layout as soon as it is
// queued (the regrouped tiles in the spare set become the bins), so that the
// next step can be queued before its flags are known; a second call undoes it.
static void commit_regroup(pic_t *h) {
    for (int s = 0; s < h->nsp; ++s) {
        SpeciesBuf &S = h->sp[s];
        S.scur ^= 1;
        const int b = S.bins;
        S.bins = S.spare;
        S.spare = b;
    }
}

// The pending step's flags (page-locked copy), after its event.
static int pending_flags(pic_t *h, int32_t *f) {
    const int p = h->pending_p;
    cudaError_t e = cudaEventSynchronize(h->ev_flags[p]);
    h->flags_pending = false;
    if (e != cudaSuccess) {
        set_error("step flags: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    *f = h->h_step_flags[4 * p];
    return flag_error(h->h_step_flags[4 * p + 1]);
}

// Regroup every species with the full sort from the pending step's push-time
// counts and its mirror (the per-tile regroup's output is dropped); the
// layout must be the one that push left.
static int rebuild_from_step(pic_t *h) {
    int64_t l0 = h->timing.launches[4];
    timing_begin(h);
    for (int s = 0; s < h->nsp; ++s)
        if (int rc = rebuild_species(h, s, REBUILD_FROM_STEP, 0)) return rc;
    timing_end(h, 1, (int)(h->timing.launches[4] - l0));
    h->rebuilds += 1;
    return 0;
}

// Finish the last step's regroup: wait for its flags and, if a bin overflowed
// or a particle moved farther than a neighbour tile, undo the commit and
// regroup with the full sort (*rebuilt set).
static int resolve_pending(pic_t *h, bool *rebuilt = nullptr) {
    if (rebuilt) *rebuilt = false;
    if (!h->flags_pending) return 0;
    int32_t f = 0;
    if (int rc = pending_flags(h, &f)) return rc;
    if (f & 3) {
        commit_regroup(h);   // back to the layout the push left
        if (int rc = rebuild_from_step(h)) return rc;
        if (rebuilt) *rebuilt = true;
    }
    return 0;
}

static int redeposit(pic_t *h) {
    if (int rc = clear_moments(h)) return rc;
    for (int s = 0; s < h->nsp; ++s)
        if (int rc = deposit_only(h, s)) return rc;
    h->moments_stale = false;
    return h->det ? fix_to_moments(h) : cell_moments(h, true);
}

// The previous step's regroup, then the moments at rest if a load or a field
// overwrite has made them stale (one deposit however many loads preceded).
static int settle(pic_t *h) {
    if (int rc = resolve_pending(h)) return rc;
    return h->moments_stale ? redeposit(h) : 0;
}

static int destroy_impl(pic_t *h) {
    if (!h) return 0;
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->st2) cudaStreamSynchronize(h->st2);
    if (h->st3) cudaStreamSynchronize(h->st3);
    if (h->pf_st) cudaStreamSynchronize(h->pf_st);
    for (pic_t::Prefetch &f : h->pf) {
        cudaFree(f.buf);
        if (f.copied) cudaEventDestroy(f.copied);
        if (f.freed) cudaEventDestroy(f.freed);
    }
    if (h->pf_st) cudaStreamDestroy(h->pf_st);
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) free_species(h->sp[s]);
    void *bufs[] = {h->E[0], h->E[1], h->H[0], h->H[1], h->Ehalf, h->B[0], h->B[1], h->M, h->Mlo, h->Mfix, h->Mc, h->cn,
                    h->cn_red, h->cn_out, h->d_removed, h->d_flags, h->d_step_flags, h->keys[0], h->keys[1],
                    h->vals[0], h->vals[1], h->hist, h->stage, h->d_diag, h->chunk_prefix, h->ticket,
                    h->d_bad, h->scan_sums, h->occ, h->touched, h->touch_list, h->rg_list, h->list_n,
                    h->ion_cell, h->ion_val, h->ion_dcell, h->ion_dval};
    for (void *p : bufs) cudaFree(p);
    if (h->h_step_flags) cudaFreeHost(h->h_step_flags);
    if (h->h_diag) cudaFreeHost(h->h_diag);
    for (cudaEvent_t ev : h->ev_flags)
        if (ev) cudaEventDestroy(ev);
    if (h->ev_batch) cudaEventDestroy(h->ev_batch);
    if (h->ev_load) cudaEventDestroy(h->ev_load);
    if (h->ev_push) cudaEventDestroy(h->ev_push);
    if (h->ev_field) cudaEventDestroy(h->ev_field);
    if (h->ev_cellm) cudaEventDestroy(h->ev_cellm);
    for (cudaEvent_t ev : h->ev_conv)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->ev_sorted)
        if (ev) cudaEventDestroy(ev);
    if (h->ev_sorts) cudaEventDestroy(h->ev_sorts);
    if (h->st2) cudaStreamDestroy(h->st2);
    if (h->st3) cudaStreamDestroy(h->st3);
    tile_free(h);
    tstate_free(h);
    delete h;
    return 0;
}

}  // namespace pic

using namespace pic;

// --------------------------------------------------------------------------- C ABI

extern "C" PIC_API const char *pic_last_error(void) { return g_err; }

// Configuration checks shared by pic_init and pic_estimate_bytes.
static int validate_config(const pic_config &c) {
    if (c.nx < 2 || c.ny < 2 || !(c.dx > 0) || !(c.dy > 0) || !(c.dt > 0)) {
        set_error("pic_init: need nx, ny >= 2 and dx, dy, dt > 0");
        return PIC_ERR_ARG;
    }
    if ((int64_t)c.nx * c.ny > (1ll << 30)) {
        set_error("pic_init: grid too large (cell index is int32)");
        return PIC_ERR_ARG;
    }
    if (c.bc_x != PIC_BC_PERIODIC && c.bc_x != PIC_BC_ABSORBING) {
        set_error("pic_init: bc_x must be PIC_BC_PERIODIC or PIC_BC_ABSORBING");
        return PIC_ERR_ARG;
    }
    if (c.cn_precond < PIC_CN_PRECOND_AUTO || c.cn_precond > PIC_CN_PRECOND_FFT) {
        set_error("pic_init: cn_precond must be PIC_CN_PRECOND_AUTO, _JACOBI or _FFT");
        return PIC_ERR_ARG;
    }
    if (c.shape < 0 || c.shape > PIC_SHAPE_QUARTIC) {
        set_error("pic_init: shape must be 0 (linear) or 1..4 (PIC_SHAPE_LINEAR .. PIC_SHAPE_QUARTIC)");
        return PIC_ERR_ARG;
    }
    if (c.field_mode != PIC_FIELD_LITERAL && c.field_mode != PIC_FIELD_CN) {
        set_error("pic_init: unknown field_mode");
        return PIC_ERR_ARG;
    }
    if (c.precision != PIC_FP64 && c.precision != PIC_FP32) {
        set_error("pic_init: precision must be PIC_FP64 or PIC_FP32");
        return PIC_ERR_ARG;
    }
    if (c.deposit != PIC_DEPOSIT_ATOMIC && c.deposit != PIC_DEPOSIT_DETERMINISTIC) {
        set_error("pic_init: unknown deposit mode");
        return PIC_ERR_ARG;
    }
    if (c.n_species < 1 || c.n_species > PIC_MAX_SPECIES) {
        set_error("pic_init: n_species must be 1..%d", PIC_MAX_SPECIES);
        return PIC_ERR_ARG;
    }
    for (int s = 0; s < c.n_species; ++s)
        if (!(c.m[s] > 0)) {
            set_error("pic_init: species %d has mass <= 0", s);
            return PIC_ERR_ARG;
        }
    if (c.tile_nx < 0 || c.tile_ny < 0 || c.tile_nx > 128 || c.tile_ny > 128) {
        set_error("pic_init: tile size must be 0 (default) or 1..128 cells");
        return PIC_ERR_ARG;
    }
    {
        const int tx = c.tile_nx > 0 ? c.tile_nx : 16, ty = c.tile_ny > 0 ? c.tile_ny : 16;
        if ((int64_t)(tx < c.nx ? tx : c.nx) * (ty < c.ny ? ty : c.ny) > PIC_MAX_TILE_CELLS) {
            set_error("pic_init: a tile may hold at most %d cells (the per-tile cell sort)", PIC_MAX_TILE_CELLS);
            return PIC_ERR_ARG;
        }
    }
    return 0;
}

// Grid, tile and halo geometry of a handle (no allocation).
static void setup_geometry(pic_t *h, const pic_config &c) {
    h->cfg = c;
    h->st = (cudaStream_t)c.cuda_stream;
    h->fp32 = (c.precision == PIC_FP32);
    h->rs = h->fp32 ? 4 : 8;
    h->det = (c.deposit == PIC_DEPOSIT_DETERMINISTIC);
    h->shape = c.shape > 1 ? c.shape : 1;
    h->periodic_x = (c.bc_x == PIC_BC_PERIODIC);
    h->nx = c.nx;
    h->ny = c.ny;
    h->nxn = h->periodic_x ? c.nx : c.nx + 1;
    h->nnode = (int64_t)h->nxn * c.ny;
    h->ncell = (int64_t)c.nx * c.ny;
    // deposit halo: the largest move per step is c dt / min(dx, dy) cells
    double maxmove = c.dt / (c.dx < c.dy ? c.dx : c.dy);
    h->halo = (int)ceil(maxmove);
    if (h->halo < 1) h->halo = 1;
    if (h->halo > 4) h->halo = 4;
    h->tnx = c.tile_nx > 0 ? c.tile_nx : 16;
    h->tny = c.tile_ny > 0 ? c.tile_ny : 16;
    if (h->tnx > c.nx) h->tnx = c.nx;
    if (h->tny > c.ny) h->tny = c.ny;
    h->ntx = (c.nx + h->tnx - 1) / h->tnx;
    h->nty = (c.ny + h->tny - 1) / h->tny;
    h->ntiles = h->ntx * h->nty;
    // ghost ring: a ragged last tile's deposit region reaches tile + halo nodes
    // past the last real node, and every node it can address must be present
    h->G = (h->tnx > h->tny ? h->tnx : h->tny) + h->halo + 1;
    h->nxp = h->nxn + 2 * h->G;
    h->nyp = c.ny + 2 * h->G;
    h->npad = (int64_t)h->nxp * h->nyp;
    h->nsp = c.n_species;
    for (int s = 0; s < h->nsp; ++s) {
        h->sp[s].q = c.q[s];
        h->sp[s].m = c.m[s];
    }
}

// The FP64 push with L2 reductions and the linear shape deposits into cell sums
// (13 moments x 4 sums per cell) that k_cell_moments turns into node moments.
static bool uses_cell_sums(const pic_t *h) { return !h->fp32 && !h->det && h->shape == 1; }
static size_t cell_sum_bytes(const pic_t *h) { return (size_t)NMOM * 4 * h->ncell * sizeof(double); }

// Device bytes a handle holds once n[s] particles of every species are loaded
// (all buffers at the sizes the library grows them to; CUDA's own context and
// allocation granularity not included).
static uint64_t estimate_bytes(const pic_t *h, const int64_t *n) {
    const uint64_t v4 = 4 * h->rs, nn = (uint64_t)h->nnode, nc = (uint64_t)h->ncell, np = (uint64_t)h->npad;
    uint64_t b = 2 * nn * v4 + 2 * nc * v4 + 3 * np * v4;
    b += (uint64_t)NMOM * nn * h->rs * (h->fp32 ? 2 : 1) + (h->det ? (uint64_t)NMOM * nn * 8 : 0);
    if (uses_cell_sums(h)) b += cell_sum_bytes(h);
    b += (uint64_t)h->nsp * 6 * (h->ntiles + 1) * 4 + ((uint64_t)h->nsp * h->ntiles + 1) * 4 + 256;
    b += (uint64_t)h->ntiles * 9 * 4 + 8 + (uint64_t)scan_sums_entries() * 4;   // neighbour table, load check, scan
    b += 10ull * (uint64_t)h->ntiles + 8;                                         // occupancy, touched and regroup tiles
    b += (uint64_t)diag_scratch_doubles(h->nsp, h->ntiles) * 8;
    if (h->cfg.field_mode == PIC_FIELD_CN) b += cn_bytes(h) + 6ull * 8 * 1024 * 8 + 24;
    int64_t stage = init_stage_doubles(h), maxcap = 0;
    for (int s = 0; s < h->nsp; ++s) {
        const int64_t ns = n ? n[s] : 0;
        if (ns <= 0) continue;
        const int64_t cap = slots_needed(h, ns);
        b += 3ull * cap * (4 + 6 * h->rs + (h->fp32 ? 0 : NCARRY * 8)) + (uint64_t)cap * 4 + 3ull * (cap / SEG) * 4;
        if (cap > maxcap) maxcap = cap;
        if (7 * ns > stage) stage = 7 * ns;
    }
    b += (uint64_t)(stage + stage / 4 + 1024) * 8;
    if (maxcap > 0) {
        const int64_t sc = 2 * maxcap + (2 * maxcap) / 8 + 4096;
        b += 4ull * sc * 4 + (uint64_t)sort_hist_entries(sc) * 4;
    }
    return b;
}

// Events that another stream waits on.  They keep timing enabled: measured on
// GB300, a wait on a timing-disabled event recorded on the caller's stream was
// released about 1.4 ms after the recorded work had finished.
static bool create_events(cudaEvent_t *ev, int n) {
    for (int k = 0; k < n; ++k)
        if (cudaEventCreateWithFlags(&ev[k], cudaEventDefault) != cudaSuccess) return false;
    return true;
}

extern "C" PIC_API int pic_init(const pic_config *cfg, pic_t **out) {
    g_err[0] = 0;
    if (!cfg || !out) {
        set_error("pic_init: NULL argument");
        return PIC_ERR_ARG;
    }
    *out = nullptr;
    const pic_config &c = *cfg;
    if (int rc = validate_config(c)) return rc;
    pic_t *h = new pic_t();
    setup_geometry(h, c);
    size_t v4 = 4 * h->rs;
    int rc = 0;
    for (int k = 0; k < 2 && !rc; ++k) rc = dalloc(&h->E[k], h->nnode * v4, "E");
    for (int k = 0; k < 2 && !rc; ++k) rc = dalloc(&h->H[k], h->ncell * v4, "H");
    for (int k = 0; k < 2 && !rc; ++k) rc = dalloc(&h->B[k], h->npad * v4, "B");
    if (!rc) rc = dalloc(&h->Ehalf, h->npad * v4, "Ehalf");
    if (!rc) rc = dalloc(&h->M, (size_t)NMOM * h->nnode * h->rs, "moments");
    if (!rc && h->fp32) rc = dalloc(&h->Mlo, (size_t)NMOM * h->nnode * h->rs, "moment compensation");
    if (!rc && h->det) rc = dalloc((void **)&h->Mfix, (size_t)NMOM * h->nnode * 8, "fixed-point moments");
    if (!rc && uses_cell_sums(h)) {
        rc = dalloc((void **)&h->Mc, cell_sum_bytes(h), "cell moment sums");
        if (!rc && cudaMemset(h->Mc, 0, cell_sum_bytes(h)) != cudaSuccess) rc = check_launch("cell moment sums");
    }
    if (!rc) rc = dalloc((void **)&h->d_removed, PIC_MAX_SPECIES * sizeof(int64_t), "counters");
    if (!rc) rc = dalloc((void **)&h->d_flags, sizeof(int32_t), "flags");
    if (!rc) rc = dalloc((void **)&h->d_bad, PIC_MAX_SPECIES * sizeof(unsigned long long), "load check");
    if (!rc) rc = dalloc((void **)&h->scan_sums, (size_t)scan_sums_entries() * sizeof(uint32_t), "scan scratch");
    if (!rc) rc = dalloc((void **)&h->d_step_flags, 2 * sizeof(int32_t), "flags");
    if (!rc) rc = dalloc((void **)&h->occ, (size_t)h->ntiles, "tile occupancy");
    if (!rc) rc = dalloc((void **)&h->touched, (size_t)h->ntiles, "touched tiles");
    if (!rc) rc = dalloc((void **)&h->touch_list, (size_t)h->ntiles * sizeof(int32_t), "touched tiles");
    if (!rc) rc = dalloc((void **)&h->rg_list, (size_t)h->ntiles * sizeof(int32_t), "regroup tiles");
    if (!rc) rc = dalloc((void **)&h->list_n, (2 + PIC_MAX_SPECIES) * sizeof(int32_t), "tile lists");
    size_t tb = (size_t)(h->ntiles + 1) * sizeof(int32_t);
    for (int s = 0; s < h->nsp && !rc; ++s) {
        SpeciesBuf &S = h->sp[s];
        rc = dalloc((void **)&S.bstart, tb, "bins");
        if (!rc) rc = dalloc((void **)&S.useg[0], tb, "bins");
        if (!rc) rc = dalloc((void **)&S.useg[1], tb, "bins");
        if (!rc) rc = dalloc((void **)&S.tcount, tb, "bins");
        if (!rc) rc = dalloc((void **)&S.cstart, tb, "bins");
        if (!rc) rc = dalloc((void **)&S.cend, tb, "bins");
    }
    if (!rc) rc = dalloc((void **)&h->chunk_prefix, ((size_t)h->nsp * h->ntiles + 1) * sizeof(int32_t), "work list");
    if (!rc) rc = dalloc((void **)&h->ticket, PIC_MAX_SPECIES * sizeof(int32_t), "work queue");
    h->diag_cap = diag_scratch_doubles(h->nsp, h->ntiles);
    if (!rc) rc = dalloc((void **)&h->d_diag, h->diag_cap * sizeof(double), "diagnostics");
    if (!rc && c.field_mode == PIC_FIELD_CN) {
        rc = dalloc(&h->cn, cn_bytes(h), "CN solver vectors");
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        h->cn_red_cap = nsm * 8;
        if (!rc) rc = dalloc((void **)&h->cn_red, 6 * (size_t)h->cn_red_cap * sizeof(double), "CN reductions");
        if (!rc) rc = dalloc((void **)&h->cn_out, 3 * sizeof(double), "CN status");
    }
    if (!rc && (cudaHostAlloc((void **)&h->h_step_flags, 8 * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess ||
                cudaHostAlloc(&h->h_diag, diag_record_bytes(), cudaHostAllocDefault) != cudaSuccess)) {
        cudaGetLastError();
        set_error("pinned host allocation failed");
        rc = PIC_ERR_OOM;
    }
    if (!rc && (cudaEventCreateWithFlags(&h->ev_flags[0], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_flags[1], cudaEventDisableTiming) != cudaSuccess ||
                !create_events(&h->ev_batch, 1) || !create_events(&h->ev_load, 1) ||
                !create_events(&h->ev_push, 1) || !create_events(&h->ev_field, 1) || !create_events(&h->ev_cellm, 1) ||
                !create_events(h->ev_conv, PIC_MAX_SPECIES) || !create_events(h->ev_sorted, PIC_MAX_SPECIES) ||
                !create_events(&h->ev_sorts, 1) ||
                cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&h->st3, cudaStreamNonBlocking) != cudaSuccess)) {
        cudaGetLastError();
        set_error("event creation failed");
        rc = PIC_ERR_CUDA;
    }
    if (!rc) rc = ensure_stage(h, init_stage_doubles(h));
    if (rc) {
        destroy_impl(h);
        return rc;
    }
    void *zero[] = {h->E[0], h->E[1], h->H[0], h->H[1], h->B[0], h->B[1], h->Ehalf};
    size_t zb[] = {h->nnode * v4, h->nnode * v4, h->ncell * v4, h->ncell * v4, h->npad * v4, h->npad * v4, h->npad * v4};
    for (int k = 0; k < 7; ++k) cudaMemsetAsync(zero[k], 0, zb[k], h->st);
    clear_moments(h);
    cudaMemsetAsync(h->d_removed, 0, PIC_MAX_SPECIES * sizeof(int64_t), h->st);
    cudaMemsetAsync(h->d_flags, 0, sizeof(int32_t), h->st);
    cudaMemsetAsync(h->d_step_flags, 0, 2 * sizeof(int32_t), h->st);
    for (int s = 0; s < h->nsp; ++s) init_empty_bins(h, s);
    if (h->cn_out) cudaMemsetAsync(h->cn_out, 0, 3 * sizeof(double), h->st);
    if (cudaStreamSynchronize(h->st) != cudaSuccess) {
        rc = check_launch("pic_init");
        destroy_impl(h);
        return rc ? rc : PIC_ERR_CUDA;
    }
    if ((rc = tile_setup(h))) {
        destroy_impl(h);
        return rc;
    }
    for (int s = 0; s < h->nsp; ++s)
        if (c.capacity[s] > 0) {
            if (int r = ensure_species_capacity(h, s, slots_needed(h, c.capacity[s]))) {
                destroy_impl(h);
                return r;
            }
        }
    *out = h;
    return PIC_OK;
}

extern "C" PIC_API int pic_destroy(pic_t *h) { return destroy_impl(h); }

extern "C" PIC_API int pic_estimate_bytes(const pic_config *cfg, const int64_t *n_per_species, uint64_t *bytes) {
    if (!cfg || !bytes) {
        set_error("pic_estimate_bytes: NULL argument");
        return PIC_ERR_ARG;
    }
    if (int rc = validate_config(*cfg)) return rc;
    pic_t tmp;
    setup_geometry(&tmp, *cfg);
    *bytes = estimate_bytes(&tmp, n_per_species);
    return PIC_OK;
}

// Device-readable views of one species' six host arrays: page-locked host
// memory is read by the conversion kernel in place (over the CPU-GPU link;
// *over_link set), device memory directly; false for pageable memory.
static bool direct_sources(const pic_species_data &d, const double *dsrc[6], bool *over_link = nullptr) {
    const double *src[6] = {d.x, d.y, d.ux, d.uy, d.uz, d.w};
    if (over_link) *over_link = false;
    for (int k = 0; k < 6; ++k) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, src[k]) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
            (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr)) {
            dsrc[k] = (const double *)at.devicePointer;
            if (over_link && at.type == cudaMemoryTypeHost) *over_link = true;
        } else {
            return false;
        }
    }
    return true;
}

// Whether the host may read p (false for device memory).
static bool host_readable(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;   // memory the runtime does not know: ordinary host memory
    }
    return at.type != cudaMemoryTypeDevice;
}

// Device-readable view of an int32 array (device or page-locked host memory), nullptr otherwise.
static const int32_t *device_view(const int32_t *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
        (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr))
        return (const int32_t *)at.devicePointer;
    return nullptr;
}

// Loads of several species (Section 3.2 (2)), all or nothing.  Every species'
// arrays are converted and checked on the GPU into its spare buffer set.  When
// every species that receives particles is empty, the stable regroup of one
// species (and, when the loaded species hold all the handle's particles, its
// deposit at rest) runs on the second stream while the next species' arrays
// are still crossing the CPU-GPU link, and an invalid particle found
// afterwards empties those species again; otherwise all checks complete
// before any regroup.
// cells: checkpoint form (restore): per entry the cell indices, with x, y of d
// holding the in-cell offsets; nullptr for global positions.
static int load_impl(pic_t *h, int nload, const int *species, const pic_species_data *d, const char *fn,
                     const int32_t *const *cells = nullptr) {
    bool seen[PIC_MAX_SPECIES] = {false};
    for (int e = 0; e < nload; ++e) {
        const int s = species[e];
        if (s < 0 || s >= h->nsp || seen[s] || d[e].n < 0) {
            set_error("%s: bad species index, repeated species or negative count (entry %d)", fn, e);
            return PIC_ERR_ARG;
        }
        seen[s] = true;
        if (d[e].n > 0 && (!d[e].x || !d[e].y || !d[e].ux || !d[e].uy || !d[e].uz || !d[e].w || (cells && !cells[e]))) {
            set_error("%s: NULL array (entry %d)", fn, e);
            return PIC_ERR_ARG;
        }
    }
    double wabs_before[PIC_MAX_SPECIES];
    for (int s = 0; s < h->nsp; ++s) wabs_before[s] = h->wabs[s];
    auto restore_wabs = [&]() {
        for (int s = 0; s < h->nsp; ++s) h->wabs[s] = wabs_before[s];
    };
    if (h->det) {
        for (int e = 0; e < nload; ++e) {
            if (d[e].n == 0) continue;
            // the bound is summed on the host in particle order (device arrays are copied first)
            const double *w = d[e].w;
            std::vector<double> wh;
            if (!host_readable(w)) {
                wh.resize((size_t)d[e].n);
                if (cudaMemcpy(wh.data(), w, (size_t)d[e].n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
                    restore_wabs();
                    return check_launch("weight bound readback");
                }
                w = wh.data();
            }
            double wabs = 0.0;
            for (int64_t p = 0; p < d[e].n; ++p) wabs += fabs(w[p]);
            h->wabs[species[e]] += wabs;   // bound of the deterministic deposit's fixed point
        }
        FixScale fs;
        if (int rc = fix_scale(h, &fs)) {
            restore_wabs();
            return rc;
        }
    }
    if (int rc = resolve_pending(h)) {
        restore_wabs();
        return rc;
    }
    // live counts (counted on the device unless no step ran since they were known) and capacity
    int64_t n0[PIC_MAX_SPECIES] = {0};
    bool fresh = true;
    int64_t staged = 0;
    int nwork = 0;
    for (int e = 0; e < nload; ++e) {
        const int s = species[e];
        const int64_t n = d[e].n;
        if (n == 0) continue;
        ++nwork;
        SpeciesBuf &S = h->sp[s];
        n0[e] = S.n;
        int rc = 0;
        if (!S.n_exact) rc = count_species(h, s, &n0[e]);
        if (!rc && n0[e] + n > 0x3fffffffll) {
            set_error("%s: more than 2^30 particles in a species", fn);
            rc = PIC_ERR_CAPACITY;
        }
        if (!rc) rc = ensure_species_capacity(h, s, slots_needed(h, n0[e] + n));
        if (rc) {
            restore_wabs();
            return rc;
        }
        fresh = fresh && n0[e] == 0;
        const double *dummy[6];
        if ((!direct_sources(d[e], dummy) || (cells && !device_view(cells[e]))) && 7 * n > staged) staged = 7 * n;
    }
    if (nwork == 0) {
        restore_wabs();
        return PIC_OK;
    }
    if (staged > 0)
        if (int rc = ensure_stage(h, staged)) {
            restore_wabs();
            return rc;
        }
    // When the loaded species are all the handle's particles, their moments at
    // rest are deposited on the second stream too, each after its regroup.
    bool eager = fresh;
    for (int s = 0; s < h->nsp && eager; ++s) {
        bool loaded = false;
        for (int e = 0; e < nload; ++e) loaded = loaded || (species[e] == s && d[e].n > 0);
        if (!loaded && !(h->sp[s].n == 0 && h->sp[s].n_exact)) eager = false;
    }
    bool cleared = false;
    cudaMemsetAsync(h->d_bad, 0xFF, PIC_MAX_SPECIES * sizeof(unsigned long long), h->st);
    cudaStream_t main_st = h->st;
    int rc = 0;
    // every conversion first (their grids are small: the regroups fill the rest of the GPU)
    for (int e = 0; e < nload && !rc; ++e) {
        const int s = species[e];
        const int64_t n = d[e].n;
        if (n == 0) continue;
        SpeciesBuf &S = h->sp[s];
        const double *dsrc[6];
        const int32_t *csrc = cells ? device_view(cells[e]) : nullptr;
        bool over_link = false;
        if (!direct_sources(d[e], dsrc, &over_link) || (cells && !csrc)) {
            // pageable: through the device stage (reused in stream order by the next species)
            over_link = false;
            const double *src[6] = {d[e].x, d[e].y, d[e].ux, d[e].uy, d[e].uz, d[e].w};
            for (int k = 0; k < 6 && !rc; ++k) {
                if (cudaMemcpyAsync(h->stage + k * n, src[k], n * sizeof(double), cudaMemcpyDefault, main_st) !=
                    cudaSuccess)
                    rc = check_launch("particle upload");
                dsrc[k] = h->stage + k * n;
            }
            if (cells && !rc) {
                if (cudaMemcpyAsync(h->stage + 6 * n, cells[e], n * sizeof(int32_t), cudaMemcpyDefault, main_st) !=
                    cudaSuccess)
                    rc = check_launch("particle upload");
                csrc = (const int32_t *)(h->stage + 6 * n);
            }
            if (rc) break;
        }
        // convert and check on the GPU; an invalid particle drops the whole load
        if ((rc = load_convert(h, s, S.spare, n, dsrc, h->d_bad + s, over_link, csrc))) break;
        S.n_exact = false;
        if (fresh) cudaEventRecord(h->ev_conv[s], main_st);
    }
    if (fresh && !rc) {
        // each species' sort on a third stream once it is converted (the sorts share their scratch:
        // one after another), its deposit at rest on the second once it is sorted -- a species'
        // sort runs beside the previous species' deposit
        for (int e = 0; e < nload && !rc; ++e) {
            const int s = species[e];
            if (d[e].n == 0) continue;
            h->st = h->st3;
            cudaStreamWaitEvent(h->st3, h->ev_conv[s], 0);
            rc = rebuild_species(h, s, REBUILD_FROM_LOAD, d[e].n);
            cudaEventRecord(h->ev_sorted[s], h->st3);
            if (!rc && eager) {
                // (after the first conversion, so after whatever the handle's stream ran before the load)
                h->st = h->st2;
                cudaStreamWaitEvent(h->st2, h->ev_sorted[s], 0);
                if (!cleared) {
                    rc = clear_moments(h);
                    cleared = true;
                }
                if (!rc) rc = deposit_only(h, s);
            }
        }
        cudaEventRecord(h->ev_sorts, h->st3);
        cudaStreamWaitEvent(h->st2, h->ev_sorts, 0);
        h->st = h->st2;
        if (!rc && eager) rc = h->det ? fix_to_moments(h) : cell_moments(h, true);
        h->st = main_st;
    }
    if (fresh) {
        cudaEventRecord(h->ev_load, h->st2);
        cudaStreamWaitEvent(main_st, h->ev_load, 0);
    }
    unsigned long long *bad = (unsigned long long *)h->h_diag;   // page-locked; diagnostics use it only inside their call
    if (!rc && (cudaMemcpyAsync(bad, h->d_bad, h->nsp * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                main_st) != cudaSuccess ||
                (fresh && cudaMemcpyAsync(h->h_step_flags + 2, h->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                          main_st) != cudaSuccess) ||
                cudaStreamSynchronize(main_st) != cudaSuccess))
        rc = check_launch("particle load check");
    int bad_e = -1;
    for (int e = 0; e < nload && !rc && bad_e < 0; ++e)
        if (d[e].n > 0 && bad[species[e]] != ~0ull) bad_e = e;
    if (rc || bad_e >= 0) {
        h->moments_stale = true;
        if (fresh)
            for (int e = 0; e < nload; ++e) {
                if (d[e].n == 0) continue;
                SpeciesBuf &S = h->sp[species[e]];
                init_empty_bins(h, species[e]);
                S.n = 0;
                S.n_exact = true;
            }
        restore_wabs();
        if (rc) return rc;
        const pic_species_data &b = d[bad_e];
        const double Lx = h->nx * h->cfg.dx, Ly = h->ny * h->cfg.dy;
        const int64_t p = (int64_t)bad[species[bad_e]];
        const double *arr[6] = {b.x, b.y, b.ux, b.uy, b.uz, b.w};
        double q[6];
        for (int k = 0; k < 6; ++k)   // host or device arrays
            if (cudaMemcpy(&q[k], arr[k] + p, sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
                cudaGetLastError();
                q[k] = NAN;
            }
        if (cells) {
            int32_t c = -1;
            if (cudaMemcpy(&c, cells[bad_e] + p, sizeof(int32_t), cudaMemcpyDefault) != cudaSuccess) cudaGetLastError();
            set_error("%s: species %d particle %lld: cell %d, offsets (%g, %g), u (%g, %g, %g), w %g: cell outside "
                      "[0,%lld), an offset outside [0,1) or a value not finite", fn, species[bad_e], (long long)p, c,
                      q[0], q[1], q[2], q[3], q[4], q[5], (long long)h->nx * h->ny);
        } else {
            set_error("%s: species %d particle %lld at (%g, %g), u (%g, %g, %g), w %g: outside [0,%g) x [0,%g) or "
                      "not finite", fn, species[bad_e], (long long)p, q[0], q[1], q[2], q[3], q[4], q[5], Lx, Ly);
        }
        return PIC_ERR_ARG;
    }
    if (!fresh)
        for (int e = 0; e < nload; ++e)
            if (d[e].n > 0)
                if (int r = rebuild_species(h, species[e], REBUILD_FROM_LOAD, d[e].n)) return r;
    h->moments_stale = !eager;   // else deposited at the next step or readout
    if (!fresh && (cudaMemcpyAsync(h->h_step_flags + 2, h->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   main_st) != cudaSuccess ||
                   cudaStreamSynchronize(main_st) != cudaSuccess))
        return check_launch(fn);
    if (int r = flag_error(h->h_step_flags[2])) return r;
    for (int e = 0; e < nload; ++e) {
        if (d[e].n == 0) continue;
        SpeciesBuf &S = h->sp[species[e]];
        S.n = n0[e] + d[e].n;
        S.n_exact = true;
    }
    return PIC_OK;
}

extern "C" PIC_API int pic_load_particles(pic_t *h, int species, int64_t n, const double *x, const double *y,
                                          const double *ux, const double *uy, const double *uz, const double *w) {
    if (!h) {
        set_error("pic_load_particles: NULL handle");
        return PIC_ERR_ARG;
    }
    pic_species_data d{n, x, y, ux, uy, uz, w};
    return load_impl(h, 1, &species, &d, "pic_load_particles");
}

extern "C" PIC_API int pic_restore_particles(pic_t *h, int species, int64_t n, const int32_t *cell, const double *ox,
                                             const double *oy, const double *ux, const double *uy, const double *uz,
                                             const double *w) {
    if (!h) {
        set_error("pic_restore_particles: NULL handle");
        return PIC_ERR_ARG;
    }
    pic_species_data d{n, ox, oy, ux, uy, uz, w};
    const int32_t *cells[1] = {cell};
    return load_impl(h, 1, &species, &d, "pic_restore_particles", cells);
}

// Field ionisation pass: decisions and staging per chain (pic_ionize.cu), then
// one load of the ionised particles into the target and electron species in
// the checkpoint form (exact cells and offsets), chain by chain in chain order.
extern "C" PIC_API int pic_ionize(pic_t *h, const pic_ionization *p, int64_t *n_ionized) {
    if (n_ionized) *n_ionized = 0;
    if (!h || !p || p->n_chains < 1 || p->n_chains >= PIC_MAX_SPECIES || !(p->field_unit_au > 0) ||
        !(p->time_unit_au > 0)) {
        set_error("pic_ionize: NULL argument, chain count outside 1..%d or non-positive unit", PIC_MAX_SPECIES - 1);
        return PIC_ERR_ARG;
    }
    if (h->shape != 1) {
        set_error("pic_ionize: the ionisation pass gathers |E| with the linear shape; the run uses shape order %d",
                  h->shape);
        return PIC_ERR_ARG;
    }
    bool ion_seen[PIC_MAX_SPECIES] = {false};
    for (int c = 0; c < p->n_chains; ++c) {
        const int a = p->ion[c], t = p->target[c], e = p->electron[c];
        if (a < 0 || a >= h->nsp || t < 0 || t >= h->nsp || e < 0 || e >= h->nsp || a == t || a == e || t == e ||
            ion_seen[a] || !(p->ip_ev[c] > 0) || h->sp[t].q - h->sp[a].q != 1.0 || h->sp[t].q <= 0) {
            set_error("pic_ionize: bad chain %d (species, repeated ion species, potential, or target charge not "
                      "the ion's plus one)", c);
            return PIC_ERR_ARG;
        }
        ion_seen[a] = true;
    }
    if (int rc = settle(h)) return rc;
    int64_t counts[PIC_MAX_SPECIES] = {0}, total = 0;
    for (int c = 0; c < p->n_chains; ++c) {
        if (int rc = count_species(h, p->ion[c], &counts[c])) return rc;
        total += counts[c];
    }
    if (total == 0) return PIC_OK;
    if (total > h->ion_cap) {
        cudaFree(h->ion_cell);
        cudaFree(h->ion_val);
        h->ion_cell = nullptr;
        h->ion_val = nullptr;
        h->ion_cap = 0;
        if (int rc = dalloc((void **)&h->ion_cell, (size_t)total * sizeof(int32_t), "ionisation staging")) return rc;
        if (int rc = dalloc((void **)&h->ion_val, (size_t)6 * total * sizeof(double), "ionisation staging")) return rc;
        h->ion_cap = total;
    }
    const double HARTREE_EV = 27.211386245988;
    int64_t off[PIC_MAX_SPECIES] = {0}, nc[PIC_MAX_SPECIES] = {0}, done = 0;
    for (int c = 0; c < p->n_chains; ++c) {
        const double ip = p->ip_ev[c] / HARTREE_EV, Z = h->sp[p->target[c]].q;
        const double n = Z / sqrt(2.0 * ip), K = 2.0 * pow(2.0 * ip, 1.5);
        IonChain ch;
        ch.species = p->ion[c];
        ch.c2ip = pow(2.0, 2.0 * n) / (n * tgamma(2.0 * n)) * ip;
        ch.expo = 2.0 * n - 1.0;
        ch.K = K;
        ch.fmax = (n > 0.5) ? K / (3.0 * (2.0 * n - 1.0)) : INFINITY;
        ch.field_au = p->field_unit_au;
        ch.dt_au = h->cfg.dt * p->time_unit_au;
        off[c] = done;
        if (int rc = ion_chain(h, ch, p->seed, h->ion_cell, h->ion_val, h->ion_cap, done, &nc[c])) return rc;
        done += nc[c];
        h->sp[p->ion[c]].n = counts[c] - nc[c];
        h->sp[p->ion[c]].n_exact = true;
    }
    if (done == 0) return PIC_OK;
    // destinations: each target and electron species, its sources in chain order
    int dest[PIC_MAX_SPECIES], ndest = 0;
    int64_t dn[PIC_MAX_SPECIES] = {0}, dsrc_count[PIC_MAX_SPECIES] = {0};
    auto add_dest = [&](int s) {
        for (int k = 0; k < ndest; ++k)
            if (dest[k] == s) return k;
        dest[ndest] = s;
        return ndest++;
    };
    for (int c = 0; c < p->n_chains; ++c) {
        if (!nc[c]) continue;
        for (int s : {p->target[c], p->electron[c]}) {
            const int k = add_dest(s);
            dn[k] += nc[c];
            dsrc_count[k] += 1;
        }
    }
    int64_t multi = 0;
    for (int k = 0; k < ndest; ++k)
        if (dsrc_count[k] > 1) multi += dn[k];
    if (multi > h->ion_dcap) {
        cudaFree(h->ion_dcell);
        cudaFree(h->ion_dval);
        h->ion_dcell = nullptr;
        h->ion_dval = nullptr;
        h->ion_dcap = 0;
        if (int rc = dalloc((void **)&h->ion_dcell, (size_t)multi * sizeof(int32_t), "ionisation staging")) return rc;
        if (int rc = dalloc((void **)&h->ion_dval, (size_t)6 * multi * sizeof(double), "ionisation staging")) return rc;
        h->ion_dcap = multi;
    }
    pic_species_data data[PIC_MAX_SPECIES];
    const int32_t *cells[PIC_MAX_SPECIES];
    int64_t moff = 0;
    const int64_t S = h->ion_cap, D = h->ion_dcap;
    for (int k = 0; k < ndest; ++k) {
        const int s = dest[k];
        if (dsrc_count[k] == 1) {
            int c = 0;
            while (!(nc[c] && (p->target[c] == s || p->electron[c] == s))) ++c;
            const double *v = h->ion_val + off[c];
            data[k] = pic_species_data{nc[c], v, v + S, v + 2 * S, v + 3 * S, v + 4 * S, v + 5 * S};
            cells[k] = h->ion_cell + off[c];
            continue;
        }
        int64_t pos = moff;
        for (int c = 0; c < p->n_chains; ++c) {
            if (!nc[c] || (p->target[c] != s && p->electron[c] != s)) continue;
            cudaMemcpyAsync(h->ion_dcell + pos, h->ion_cell + off[c], nc[c] * sizeof(int32_t),
                            cudaMemcpyDeviceToDevice, h->st);
            for (int q = 0; q < 6; ++q)
                cudaMemcpyAsync(h->ion_dval + (int64_t)q * D + pos, h->ion_val + (int64_t)q * S + off[c],
                                nc[c] * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
            pos += nc[c];
        }
        const double *v = h->ion_dval + moff;
        data[k] = pic_species_data{dn[k], v, v + D, v + 2 * D, v + 3 * D, v + 4 * D, v + 5 * D};
        cells[k] = h->ion_dcell + moff;
        moff = pos;
    }
    if (int rc = check_launch("ionisation staging copies")) return rc;
    if (int rc = load_impl(h, ndest, dest, data, "pic_ionize", cells)) return rc;
    if (n_ionized) *n_ionized = done;
    return PIC_OK;
}

extern "C" PIC_API int pic_collide(pic_t *h, const pic_collisions *p, int64_t *n_pairs) {
    if (n_pairs) *n_pairs = 0;
    if (!h || !p || p->n_pairs < 1 || p->n_pairs > PIC_MAX_COLLISION_PAIRS || !(p->ln_lambda > 0) ||
        !(p->kappa > 0)) {
        set_error("pic_collide: NULL argument, entry count outside 1..%d or non-positive ln_lambda / kappa",
                  PIC_MAX_COLLISION_PAIRS);
        return PIC_ERR_ARG;
    }
    for (int k = 0; k < p->n_pairs; ++k)
        if (p->a[k] < 0 || p->a[k] >= h->nsp || p->b[k] < 0 || p->b[k] >= h->nsp) {
            set_error("pic_collide: entry %d names a species outside 0..%d", k, h->nsp - 1);
            return PIC_ERR_ARG;
        }
    if (int rc = settle(h)) return rc;
    unsigned long long *d = nullptr;
    if (cudaMallocAsync((void **)&d, sizeof(unsigned long long), h->st) != cudaSuccess) {
        cudaGetLastError();
        set_error("pic_collide: allocation failed");
        return PIC_ERR_OOM;
    }
    cudaMemsetAsync(d, 0, sizeof(unsigned long long), h->st);
    int rc = collide(h, p, d);
    unsigned long long total = 0;
    if (!rc && (cudaMemcpyAsync(&total, d, sizeof(total), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
                cudaStreamSynchronize(h->st) != cudaSuccess))
        rc = check_launch("pic_collide");
    cudaFreeAsync(d, h->st);
    // u changed: the moments (and, FP64 form, the carried 1/gamma, b, 1/(1+|b|^2)) are redeposited at rest
    h->moments_stale = true;
    if (rc) return rc;
    if (n_pairs) *n_pairs = (int64_t)total;
    return PIC_OK;
}

extern "C" PIC_API int pic_set_step(pic_t *h, int64_t step) {
    if (!h || step < 0) {
        set_error("pic_set_step: NULL handle or negative step");
        return PIC_ERR_ARG;
    }
    if (int rc = resolve_pending(h)) return rc;
    h->step = step;
    return PIC_OK;
}

extern "C" PIC_API int pic_load_species(pic_t *h, int nspecies, const pic_species_data *data) {
    if (!h || nspecies < 0 || (nspecies > 0 && !data)) {
        set_error("pic_load_species: NULL handle or data, or negative species count");
        return PIC_ERR_ARG;
    }
    if (nspecies > h->nsp) {
        set_error("pic_load_species: %d species given, the handle has %d", nspecies, h->nsp);
        return PIC_ERR_ARG;
    }
    int idx[PIC_MAX_SPECIES];
    for (int s = 0; s < nspecies; ++s) idx[s] = s;
    return load_impl(h, nspecies, idx, data, "pic_load_species");
}

extern "C" PIC_API int pic_prefetch_species(pic_t *h, int nspecies, const pic_species_data *data) {
    if (!h || nspecies < 0 || (nspecies > 0 && !data)) {
        set_error("pic_prefetch_species: NULL handle or data, or negative species count");
        return PIC_ERR_ARG;
    }
    if (nspecies > h->nsp) {
        set_error("pic_prefetch_species: %d species given, the handle has %d", nspecies, h->nsp);
        return PIC_ERR_ARG;
    }
    int64_t total = 0;
    for (int s = 0; s < nspecies; ++s) {
        const pic_species_data &d = data[s];
        if (d.n < 0 || (d.n > 0 && (!d.x || !d.y || !d.ux || !d.uy || !d.uz || !d.w))) {
            set_error("pic_prefetch_species: negative count or NULL array (species %d)", s);
            return PIC_ERR_ARG;
        }
        total += 6 * d.n;
    }
    if (h->pf_count == 2) {
        set_error("pic_prefetch_species: two prefetched loads are waiting already");
        return PIC_ERR_STATE;
    }
    if (!h->pf_st && cudaStreamCreateWithFlags(&h->pf_st, cudaStreamNonBlocking) != cudaSuccess)
        return check_launch("prefetch stream");
    pic_t::Prefetch &f = h->pf[(h->pf_head + h->pf_count) & 1];
    if ((!f.copied && cudaEventCreateWithFlags(&f.copied, cudaEventDisableTiming) != cudaSuccess) ||
        (!f.freed && cudaEventCreateWithFlags(&f.freed, cudaEventDisableTiming) != cudaSuccess))
        return check_launch("prefetch events");
    if (total > f.cap) {
        // the slot's last load has returned, but its copies may be in flight on an error path
        cudaStreamSynchronize(h->pf_st);
        cudaFree(f.buf);
        f.buf = nullptr;
        f.cap = 0;
        if (cudaMalloc(&f.buf, (size_t)total * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            set_error("pic_prefetch_species: out of device memory (%lld bytes)", (long long)(total * 8));
            return PIC_ERR_OOM;
        }
        f.cap = total;
    }
    cudaStreamWaitEvent(h->pf_st, f.freed, 0);   // the slot's previous load has read its copy
    int64_t off = 0;
    for (int s = 0; s < nspecies; ++s) {
        const pic_species_data &d = data[s];
        const double *src[6] = {d.x, d.y, d.ux, d.uy, d.uz, d.w};
        for (int k = 0; k < 6 && d.n > 0; ++k) {
            if (cudaMemcpyAsync(f.buf + off, src[k], (size_t)d.n * sizeof(double), cudaMemcpyDefault, h->pf_st) !=
                cudaSuccess)
                return check_launch("prefetch copy");
            off += d.n;
        }
        f.n[s] = d.n;
    }
    f.nsp = nspecies;
    cudaEventRecord(f.copied, h->pf_st);
    h->pf_count += 1;
    return check_launch("pic_prefetch_species");
}

extern "C" PIC_API int pic_load_prefetched(pic_t *h) {
    if (!h) return PIC_ERR_ARG;
    if (h->pf_count == 0) {
        set_error("pic_load_prefetched: nothing is prefetched");
        return PIC_ERR_STATE;
    }
    pic_t::Prefetch &f = h->pf[h->pf_head];
    h->pf_head ^= 1;
    h->pf_count -= 1;
    pic_species_data sd[PIC_MAX_SPECIES];
    int idx[PIC_MAX_SPECIES];
    int64_t off = 0;
    for (int s = 0; s < f.nsp; ++s) {
        const int64_t n = f.n[s];
        const double *b = f.buf + off;
        sd[s] = pic_species_data{n, b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n};
        idx[s] = s;
        off += 6 * n;
    }
    cudaStreamWaitEvent(h->st, f.copied, 0);   // on the GPU: the load's conversions read the copy
    if (h->det) cudaEventSynchronize(f.copied);   // the exact deposit's weight bound reads the weights on the host
    const int rc = load_impl(h, f.nsp, idx, sd, "pic_load_prefetched");
    cudaEventRecord(f.freed, h->st);
    return rc;
}

extern "C" PIC_API int pic_clear_particles(pic_t *h) {
    if (!h) return PIC_ERR_ARG;
    if (int rc = resolve_pending(h)) return rc;
    for (int s = 0; s < h->nsp; ++s) {
        init_empty_bins(h, s);
        h->sp[s].n = 0;
        h->sp[s].n_exact = true;
        h->wabs[s] = 0.0;
    }
    if (int rc = clear_moments(h)) return rc;
    h->moments_stale = false;
    return cudaStreamSynchronize(h->st) == cudaSuccess ? PIC_OK : check_launch("pic_clear_particles");
}

// A step's flags word (parity p) zeroed, the tile lists reset and, if asked,
// the push's work items built from the current layout.
static int step_reset(pic_t *h, int p, bool prep) {
    cudaMemsetAsync(h->d_step_flags + p, 0, sizeof(int32_t), h->st);
    if (int rc = reset_lists(h)) return rc;
    return prep ? push_prep(h, false) : 0;
}

// The particle part of a step (parity p): push (+ the exact deposit's
// conversion), touch map, the FP64 cell sums into node moments (on the field
// stream when it overlaps), regroup, and the flags copied to the host.  guard:
// the previous step's flags word; the kernels do nothing if it holds a failure.
static int particle_step(pic_t *h, int p, const int32_t *guard, cudaStream_t main_st, bool overlap) {
    h->guard = guard;
    struct Reset {
        pic_t *h;
        ~Reset() { h->guard = nullptr; }
    } reset{h};
    timing_begin(h);
    int64_t l0 = h->timing.launches[4];
    if (int rc = particle_tiles(h, true)) return rc;
    if (h->det)
        if (int rc = fix_to_moments(h)) return rc;
    timing_end(h, 0, (int)(h->timing.launches[4] - l0));
    // node tiles this deposit may have written: read by the next field solve and cleared before the next push
    if (int rc = touch_map(h)) return rc;
    h->touch_all = false;
    if (overlap) cudaEventRecord(h->ev_push, main_st);
    // the FP64 push's cell sums into the node moments (beside the regroup; before the next field solve)
    if (h->Mc) {
        if (overlap) {
            cudaStreamWaitEvent(h->st2, h->ev_push, 0);
            h->st = h->st2;
        }
        int rc = cell_moments(h);
        if (overlap) {
            cudaEventRecord(h->ev_cellm, h->st2);
            h->st = main_st;
        }
        if (rc) return rc;
    }
    // per-tile regroup: stayers and arrivals, stably by cell, into the spare set
    timing_begin(h);
    if (int rc = regroup_tiles(h)) return rc;
    timing_end(h, 1, 1);
    cudaMemcpyAsync(h->h_step_flags + 4 * p, h->d_step_flags + p, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    cudaMemcpyAsync(h->h_step_flags + 4 * p + 1, h->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    cudaEventRecord(h->ev_flags[p], h->st);
    if (overlap && h->Mc) cudaStreamWaitEvent(main_st, h->ev_cellm, 0);   // later work reads the node moments
    return 0;
}

extern "C" PIC_API int pic_step(pic_t *h, int nsteps) {
    if (!h || nsteps < 0) {
        set_error("pic_step: bad handle or step count");
        return PIC_ERR_ARG;
    }
    if (nsteps > 0 && h->moments_stale) {
        if (int rc = settle(h)) return rc;
    }
    // The literal field solve runs on the second stream beside the previous step's regroup: it
    // needs the moments and fields the previous push left (and rewrites the E^{n+1/2} and node B
    // that push read), not its particles.  The CN solve, a cooperative kernel whose blocks wait on
    // one another, stays on the handle's stream.
    cudaStream_t main_st = h->st;
    const bool overlap = h->cfg.field_mode == PIC_FIELD_LITERAL;
    if (overlap) cudaEventRecord(h->ev_push, main_st);   // what is queued so far
    bool prepped = false;   // the push's work items of this step are queued
    for (int k = 0; k < nsteps; ++k) {
        // 1. field solve (Eqs. 4-5), node B of the new H, ghost rings
        if (overlap) {
            cudaStreamWaitEvent(h->st2, h->ev_push, 0);
            h->st = h->st2;
        }
        timing_begin(h);
        int64_t l0 = h->timing.launches[4];
        int rc = overlap ? field_literal(h) : field_cn(h);
        if (!rc) rc = node_average(h, 1 - h->hcur, 1 - h->bcur);
        if (!rc) rc = fill_ghosts(h, h->Ehalf);
        if (!rc) timing_end(h, 2, (int)(h->timing.launches[4] - l0));
        if (overlap) {
            // whatever the handle's stream runs next (the push, a rebuild, or the next call after an
            // error) comes after the field solve
            cudaEventRecord(h->ev_field, h->st2);
            h->st = main_st;
            cudaStreamWaitEvent(main_st, h->ev_field, 0);
        }
        if (rc) return rc;
        // 2. the moments the field solve has read cleared (the literal solve zeroes them itself), this
        //    step's flags and the tile lists reset, and the push's work items (unless the previous step
        //    queued them behind its regroup)
        const int p = (int)(h->step & 1);
        timing_begin(h);
        l0 = h->timing.launches[4];
        if ((rc = clear_step_moments(h))) return rc;
        if ((rc = step_reset(h, p, !prepped))) return rc;
        prepped = false;
        timing_end(h, 3, (int)(h->timing.launches[4] - l0));
        // 3. push, deposit, regroup -- queued at once: they do nothing if the previous step's regroup
        //    (still in flight) fails, and the host redoes them after the full sort below
        const bool prev = h->flags_pending;
        if ((rc = particle_step(h, p, prev ? h->d_step_flags + (1 - p) : nullptr, main_st, overlap))) return rc;
        commit_regroup(h);
        if (prev) {
            // the previous step's regroup decision (the host waits for its flags while the GPU works)
            int32_t f = 0;
            if ((rc = pending_flags(h, &f))) return rc;
            if (f & 3) {
                // this step's particle kernels did nothing and its commit undid the previous one: the
                // layout is the one the previous push left
                cudaMemsetAsync(h->d_step_flags + (1 - p), 0, sizeof(int32_t), h->st);
                if ((rc = rebuild_from_step(h))) return rc;
                if ((rc = step_reset(h, p, true))) return rc;
                if ((rc = particle_step(h, p, nullptr, main_st, overlap))) return rc;
                commit_regroup(h);
            }
        }
        h->flags_pending = true;
        h->pending_p = p;
        h->ecur = 1 - h->ecur;
        h->hcur = 1 - h->hcur;
        h->bcur = 1 - h->bcur;
        h->step += 1;
        for (int s = 0; s < h->nsp; ++s) h->sp[s].n_exact = false;
        // the next step's work items right behind this regroup, beside the next field solve (only
        // within this call: between calls a load or a rebuild may change the layout)
        if (k + 1 < nsteps) {
            timing_begin(h);
            l0 = h->timing.launches[4];
            if ((rc = push_prep(h, false))) return rc;
            timing_end(h, 3, (int)(h->timing.launches[4] - l0));
            prepped = true;
        }
    }
    return PIC_OK;
}

// --------------------------------------------------------------------------- batched runs

struct pic_batch {
    pic::BatchScratch b;
};

extern "C" PIC_API int pic_batch_create(int max_runs, void *cuda_stream, pic_batch **out) {
    if (!out || max_runs < 1) {
        set_error("pic_batch_create: bad argument");
        return PIC_ERR_ARG;
    }
    *out = nullptr;
    pic_batch *p = new pic_batch();
    BatchScratch &b = p->b;
    b.st = (cudaStream_t)cuda_stream;
    b.cap = max_runs;
    bool ok = cudaMalloc(&b.args_dev, (size_t)max_runs * batch_args_bytes()) == cudaSuccess &&
              cudaMalloc((void **)&b.idx, (size_t)(2 * (max_runs + 1) + 1) * sizeof(int32_t)) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
        ok = cudaHostAlloc(&b.args_host[k], (size_t)max_runs * batch_args_bytes(), cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&b.idx_host[k], (size_t)(max_runs + 1) * sizeof(int32_t), cudaHostAllocDefault) ==
                 cudaSuccess &&
             cudaEventCreateWithFlags(&b.ev_stage[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && create_events(&b.ev_push, 1) && create_events(&b.ev_done, 1);
    if (!ok) {
        cudaGetLastError();
        set_error("pic_batch_create: allocation failed");
        pic_batch_destroy(p);
        return PIC_ERR_OOM;
    }
    *out = p;
    return PIC_OK;
}

extern "C" PIC_API int pic_batch_destroy(pic_batch *p) {
    if (!p) return PIC_OK;
    BatchScratch &b = p->b;
    if (b.st) cudaStreamSynchronize(b.st);
    else cudaDeviceSynchronize();
    cudaFree(b.args_dev);
    cudaFree(b.idx);
    for (int k = 0; k < 2; ++k) {
        if (b.args_host[k]) cudaFreeHost(b.args_host[k]);
        if (b.idx_host[k]) cudaFreeHost(b.idx_host[k]);
        if (b.ev_stage[k]) cudaEventDestroy(b.ev_stage[k]);
    }
    if (b.ev_push) cudaEventDestroy(b.ev_push);
    if (b.ev_done) cudaEventDestroy(b.ev_done);
    delete p;
    return PIC_OK;
}

// Each step: every run's field solve and clears on its own stream; then one
// push launch and one regroup launch over the work items of all runs on the
// batch stream; then every run's step flags on its stream.  As in a single
// run's steps, a step is queued before the previous step's regroup decision
// is known: a run whose previous regroup failed contributes no work items and
// no regroup blocks, and the host redoes its step on the run's own stream
// after the full sort.
extern "C" PIC_API int pic_batch_step(pic_batch *p, pic_t **hs, int n, int nsteps) {
    if (!p || !hs || n < 1 || n > p->b.cap || nsteps < 0) {
        set_error("pic_batch_step: bad argument");
        return PIC_ERR_ARG;
    }
    for (int r = 0; r < n; ++r) {
        if (!hs[r] || hs[r]->fp32 != hs[0]->fp32 || hs[r]->det != hs[0]->det) {
            set_error("pic_batch_step: runs of one batch need one precision and one deposit mode");
            return PIC_ERR_ARG;
        }
        if (hs[r]->shape != 1) {
            set_error("pic_batch_step: batched steps use the linear shape (run %d has shape order %d)", r, hs[r]->shape);
            return PIC_ERR_ARG;
        }
    }
    BatchScratch &b = p->b;
    for (int r = 0; r < n; ++r)
        if (hs[r]->moments_stale)
            if (int rc = settle(hs[r])) return rc;
    std::vector<char> prev(n);
    struct Reset {
        pic_t **hs;
        int n;
        ~Reset() {
            for (int r = 0; r < n; ++r) hs[r]->guard = nullptr;
        }
    } reset{hs, n};
    for (int k = 0; k < nsteps; ++k) {
        for (int r = 0; r < n; ++r) {
            pic_t *h = hs[r];
            int rc = (h->cfg.field_mode == PIC_FIELD_LITERAL) ? field_literal(h) : field_cn(h);
            if (!rc) rc = node_average(h, 1 - h->hcur, 1 - h->bcur);
            if (!rc) rc = fill_ghosts(h, h->Ehalf);
            if (rc) return rc;
        }
        for (int r = 0; r < n; ++r) {
            pic_t *h = hs[r];
            const int ph = (int)(h->step & 1);
            prev[r] = h->flags_pending ? 1 : 0;
            h->guard = prev[r] ? h->d_step_flags + (1 - ph) : nullptr;
            if (int rc = clear_step_moments(h)) return rc;
            cudaMemsetAsync(h->d_step_flags + ph, 0, sizeof(int32_t), h->st);
            if (int rc = push_work_list(h)) return rc;
            if (int rc = reset_lists(h)) return rc;
            cudaEventRecord(h->ev_batch, h->st);
            cudaStreamWaitEvent(b.st, h->ev_batch, 0);
        }
        if (int rc = batch_push(b, hs, n)) return rc;
        if (hs[0]->det) {
            cudaEventRecord(b.ev_push, b.st);
            for (int r = 0; r < n; ++r) {
                cudaStreamWaitEvent(hs[r]->st, b.ev_push, 0);
                if (int rc = fix_to_moments(hs[r])) return rc;
            }
        }
        if (int rc = batch_regroup(b, hs, n)) return rc;
        cudaEventRecord(b.ev_done, b.st);
        for (int r = 0; r < n; ++r) {
            pic_t *h = hs[r];
            cudaStreamWaitEvent(h->st, b.ev_done, 0);
            // the run's touched tiles, as after its own push (the batched regroup visited every tile)
            if (int rc = touch_map(h)) return rc;
            h->touch_all = false;
            h->guard = nullptr;
            const int ph = (int)(h->step & 1);
            cudaMemcpyAsync(h->h_step_flags + 4 * ph, h->d_step_flags + ph, sizeof(int32_t), cudaMemcpyDeviceToHost,
                            h->st);
            cudaMemcpyAsync(h->h_step_flags + 4 * ph + 1, h->d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
            cudaEventRecord(h->ev_flags[ph], h->st);
            commit_regroup(h);
        }
        // the previous step's regroup decisions (the host waits for their flags while the GPU works)
        for (int r = 0; r < n; ++r) {
            if (!prev[r]) continue;
            pic_t *h = hs[r];
            const int ph = (int)(h->step & 1);
            int32_t f = 0;
            if (int rc = pending_flags(h, &f)) return rc;
            if (f & 3) {
                // this step did nothing for the run and its commit undid the previous one: the layout is
                // the one the previous push left; the full sort, then the step alone on the run's stream
                cudaMemsetAsync(h->d_step_flags + (1 - ph), 0, sizeof(int32_t), h->st);
                if (int rc = rebuild_from_step(h)) return rc;
                if (int rc = step_reset(h, ph, true)) return rc;
                if (int rc = particle_step(h, ph, nullptr, h->st, false)) return rc;
                commit_regroup(h);
            }
        }
        for (int r = 0; r < n; ++r) {
            pic_t *h = hs[r];
            h->flags_pending = true;
            h->pending_p = (int)(h->step & 1);
            h->ecur = 1 - h->ecur;
            h->hcur = 1 - h->hcur;
            h->bcur = 1 - h->bcur;
            h->step += 1;
            for (int s = 0; s < h->nsp; ++s) h->sp[s].n_exact = false;
        }
    }
    return PIC_OK;
}

extern "C" PIC_API int pic_sync(pic_t *h) {
    if (!h) return PIC_ERR_ARG;
    if (int rc = settle(h)) return rc;
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        set_error("pic_sync: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return check_launch("pic_sync");
}

extern "C" PIC_API int pic_moments(pic_t *h, double *rho, double *S9, double *dj3) {
    if (!h) return PIC_ERR_ARG;
    if (int rc = settle(h)) return rc;
    // area-normalised FP64 planes made on the device, then copied straight into the caller's arrays
    if (int rc = ensure_stage(h, (int64_t)NMOM * h->nnode)) return rc;
    if (int rc = moments_to_stage(h)) return rc;
    const size_t n = (size_t)h->nnode * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (rho) e = cudaMemcpyAsync(rho, h->stage, n, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && S9) e = cudaMemcpyAsync(S9, h->stage + h->nnode, 9 * n, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess && dj3)
        e = cudaMemcpyAsync(dj3, h->stage + 10 * h->nnode, 3 * n, cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        set_error("pic_moments: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}

extern "C" PIC_API int pic_fields(pic_t *h, double *E3, double *H3) {
    if (!h) return PIC_ERR_ARG;
    if (int rc = resolve_pending(h)) return rc;
    return download_fields(h, E3, H3);
}

extern "C" PIC_API int pic_set_fields(pic_t *h, const double *E3, const double *H3) {
    if (!h) return PIC_ERR_ARG;
    if (int rc = resolve_pending(h)) return rc;
    if (int rc = upload_fields(h, E3, H3)) return rc;
    if (int rc = node_average(h, h->hcur, h->bcur)) return rc;
    h->moments_stale = true;
    return cudaStreamSynchronize(h->st) == cudaSuccess ? PIC_OK : check_launch("pic_set_fields");
}

extern "C" PIC_API int pic_particle_count(pic_t *h, int species, int64_t *n) {
    if (!h || !n || species < 0 || species >= h->nsp) {
        set_error("pic_particle_count: bad argument");
        return PIC_ERR_ARG;
    }
    if (int rc = resolve_pending(h)) return rc;
    return count_species(h, species, n);
}

extern "C" PIC_API int pic_get_particles(pic_t *h, int species, double *x, double *y, double *ux, double *uy, double *uz,
                                 double *w, int32_t *cell) {
    if (!h || species < 0 || species >= h->nsp) {
        set_error("pic_get_particles: bad argument");
        return PIC_ERR_ARG;
    }
    if (int rc = resolve_pending(h)) return rc;
    int64_t n = 0;
    if (int rc = particles_to_stage(h, species, &n)) return rc;
    if (n == 0) return PIC_OK;
    double *dst[6] = {x, y, ux, uy, uz, w};
    for (int k = 0; k < 6; ++k)
        if (dst[k]) cudaMemcpyAsync(dst[k], h->stage + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (cell) cudaMemcpyAsync(cell, h->stage + 6 * n, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        set_error("pic_get_particles: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}

extern "C" PIC_API int pic_save_particles(pic_t *h, int species, int32_t *cell, double *ox, double *oy, double *ux,
                                          double *uy, double *uz, double *w) {
    if (!h || species < 0 || species >= h->nsp) {
        set_error("pic_save_particles: bad argument");
        return PIC_ERR_ARG;
    }
    if (int rc = resolve_pending(h)) return rc;
    int64_t n = 0;
    if (int rc = particles_to_stage(h, species, &n, true)) return rc;
    if (n == 0) return PIC_OK;
    double *dst[6] = {ox, oy, ux, uy, uz, w};
    for (int k = 0; k < 6; ++k)
        if (dst[k]) cudaMemcpyAsync(dst[k], h->stage + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    if (cell) cudaMemcpyAsync(cell, h->stage + 6 * n, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    cudaError_t e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        set_error("pic_save_particles: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return PIC_OK;
}

extern "C" PIC_API int pic_diagnostics(pic_t *h, pic_diag *out) {
    if (!h || !out) return PIC_ERR_ARG;
    memset(out, 0, sizeof(*out));
    if (int rc = settle(h)) return rc;
    if (int rc = diagnostics(h, out)) return rc;
    out->step = h->step;
    out->full_regroups = (int32_t)h->rebuilds;
    return PIC_OK;
}

extern "C" PIC_API int pic_set_timing(pic_t *h, int enabled) {
    if (!h) return PIC_ERR_ARG;
    h->timing.enabled = enabled != 0;
    return PIC_OK;
}

extern "C" PIC_API int pic_timings(pic_t *h, double ms[4], int64_t launches[5], int reset) {
    if (!h) return PIC_ERR_ARG;
    if (int rc = harvest(h)) return rc;
    for (int k = 0; k < 4; ++k)
        if (ms) ms[k] = h->timing.ms[k];
    for (int k = 0; k < 5; ++k)
        if (launches) launches[k] = h->timing.launches[k];
    if (reset) {
        for (int k = 0; k < 4; ++k) h->timing.ms[k] = 0;
        for (int k = 0; k < 5; ++k) h->timing.launches[k] = 0;
    }
    return PIC_OK;
}
