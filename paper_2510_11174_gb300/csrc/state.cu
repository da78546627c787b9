// Checkpoint and restore of a context (hyb_get_state / hyb_set_state; see
// include/hyb.h).  The paper keeps its runs reproducible from stored
// parameters, data and fixed random streams (Methodology); a saved state plus
// the counter-based random streams (keyed by particle id and step) and the
// order-independent deposition let a restored run continue bit for bit.
//
// Layout of the byte image (host memory, native endianness), each section
// padded to 8 bytes:
//   StateHeader
//   E, B, J                     3 x 3 N FP32 (component-major, x fastest)
//   Mur history planes          24 x mur_plane FP32
//   rho_bg                      N FP32
//   mask, mask_prev             N bytes each
//   per species: SpeciesHeader, per-tile tallies (NTALLY x ntiles FP64, then
//                NTALLY x ntiles u64), then n particles as x, y, z, ux, uy,
//                uz, w (FP32), zq (FP32, if the species has charge states),
//                tau (FP32, if it has optical depths), ids (u64), tile after tile
//   per fluid:   FluidHeader, n, ux, uy, uz (N FP32 each)
#include <cstring>
#include <string>
#include <vector>

#include "hyb_internal.cuh"

namespace hyb {

static constexpr char STATE_MAGIC[8] = {'H', 'Y', 'B', 'S', 'T', 'A', 'T', '1'};
static constexpr uint32_t STATE_VERSION = 1;

struct StateHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t n[3], bc[3], T;
    uint32_t seed;
    double d[3], dt;
    int32_t n_species, n_fluids;
    long long step;
    uint32_t epoch;
    int32_t fluids_idle;
    int32_t status;
    int32_t order;
    long long mur_plane;
    uint64_t total_bytes;
    hyb_regime_desc regime;
};

struct SpeciesHeader {
    double q, m;
    int32_t kind, zmax, has_zq, has_tau;
    int32_t cap, pad;
    long long n;
};

struct FluidHeader {
    double q, m;
    unsigned long long clamped;
};

static size_t pad8(size_t b) { return (b + 7) & ~(size_t)7; }

// per-tile live counts of a species (host copy)
static hyb_status species_counts(hyb_ctx *c, const Species &sp, std::vector<int> &cnt, long long &total) {
    cnt.assign((size_t)c->g.ntiles, 0);
    HYB_CUDA_TRY(cudaMemcpyAsync(cnt.data(), sp.dev.count, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost,
                                 c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    total = 0;
    for (int &v : cnt) {
        v = std::min(v, sp.cap);
        total += v;
    }
    return HYB_OK;
}

static size_t species_bytes(const Species &sp, long long n, int ntiles) {
    size_t b = pad8(sizeof(SpeciesHeader));
    b += pad8(sizeof(double) * NTALLY * (size_t)ntiles) + pad8(sizeof(unsigned long long) * NTALLY * (size_t)ntiles);
    const int nf = 7 + (sp.dev.zq ? 1 : 0) + (sp.dev.tau ? 1 : 0);
    b += (size_t)nf * pad8(sizeof(float) * (size_t)n) + pad8(sizeof(uint64_t) * (size_t)n);
    return b;
}

// temporary device buffers: from the caller's arena (released afterwards) or cudaMalloc
struct Scratch {
    hyb_ctx *c;
    size_t mark;
    std::vector<void *> owned;
    explicit Scratch(hyb_ctx *ctx) : c(ctx), mark(ctx->arena.used) {}
    bool get(void **p, size_t bytes) {
        if (c->arena.base) return ctx_alloc(c, p, bytes) == cudaSuccess;
        if (cudaMalloc(p, bytes ? bytes : 256) != cudaSuccess) return false;
        owned.push_back(*p);
        return true;
    }
    ~Scratch() {
        cudaStreamSynchronize(c->stream);
        for (void *p : owned) cudaFree(p);
        if (c->arena.base) c->arena.used = mark;
    }
};

}  // namespace hyb

using namespace hyb;

extern "C" {

hyb_status hyb_get_state(hyb_ctx *c, void *buf, size_t cap, size_t *size_out) {
    if (!c || !size_out) return set_error(HYB_EINVAL, "null argument");
    const GridDev &g = c->g;
    const size_t N = (size_t)g.N;
    std::vector<std::vector<int>> counts(c->sp.size());
    std::vector<long long> totals(c->sp.size());
    size_t bytes = pad8(sizeof(StateHeader)) + 3 * 3 * pad8(sizeof(float) * N) +
                   pad8(sizeof(float) * 24 * (size_t)c->mur_plane) + pad8(sizeof(float) * N) + 2 * pad8(N);
    for (size_t s = 0; s < c->sp.size(); ++s) {
        hyb_status st = species_counts(c, c->sp[s], counts[s], totals[s]);
        if (st != HYB_OK) return st;
        bytes += species_bytes(c->sp[s], totals[s], g.ntiles);
    }
    bytes += c->fluids.size() * (pad8(sizeof(FluidHeader)) + 4 * pad8(sizeof(float) * N));
    *size_out = bytes;
    if (!buf) return HYB_OK;
    if (cap < bytes) return set_error(HYB_EINVAL, "state buffer too small (" + std::to_string(bytes) + " bytes needed)");
    char *out = static_cast<char *>(buf);
    size_t off = 0;
    auto put_host = [&](const void *src, size_t b) {
        std::memcpy(out + off, src, b);
        off += pad8(b);
    };
    auto put_dev = [&](const void *src, size_t b) -> cudaError_t {
        const cudaError_t e = cudaMemcpyAsync(out + off, src, b, cudaMemcpyDeviceToHost, c->stream);
        off += pad8(b);
        return e;
    };
    int status = 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));

    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, STATE_MAGIC, 8);
    h.version = STATE_VERSION;
    h.header_bytes = sizeof(StateHeader);
    for (int a = 0; a < 3; ++a) {
        h.n[a] = g.n[a];
        h.bc[a] = g.bc[a];
        h.d[a] = g.dd[a];
    }
    h.T = g.T;
    h.seed = g.seed;
    h.dt = g.dt_d;
    h.n_species = (int32_t)c->sp.size();
    h.n_fluids = (int32_t)c->fluids.size();
    h.step = c->step;
    h.epoch = c->epoch;
    h.fluids_idle = c->fluids_idle ? 1 : 0;
    h.status = status;
    h.order = g.order;
    h.mur_plane = c->mur_plane;
    h.total_bytes = bytes;
    h.regime = c->regime;
    put_host(&h, sizeof(h));
    const float *fields[3] = {c->E, c->B, c->J};
    for (const float *f : fields)
        for (int q = 0; q < 3; ++q) HYB_CUDA_TRY(put_dev(f + q * N, sizeof(float) * N));
    HYB_CUDA_TRY(put_dev(c->mur_old, sizeof(float) * 24 * (size_t)c->mur_plane));
    HYB_CUDA_TRY(put_dev(c->rho_bg, sizeof(float) * N));
    HYB_CUDA_TRY(put_dev(c->mask, N));
    HYB_CUDA_TRY(put_dev(c->mask_prev, N));

    for (size_t s = 0; s < c->sp.size(); ++s) {
        const Species &sp = c->sp[s];
        const SpDev &d = sp.dev;
        SpeciesHeader sh;
        std::memset(&sh, 0, sizeof(sh));
        sh.q = sp.q;
        sh.m = sp.m;
        sh.kind = d.kind;
        sh.zmax = d.zmax;
        sh.has_zq = d.zq ? 1 : 0;
        sh.has_tau = d.tau ? 1 : 0;
        sh.cap = sp.cap;
        sh.n = totals[s];
        put_host(&sh, sizeof(sh));
        HYB_CUDA_TRY(put_dev(d.tal_e, sizeof(double) * NTALLY * (size_t)g.ntiles));
        HYB_CUDA_TRY(put_dev(d.tal_n, sizeof(unsigned long long) * NTALLY * (size_t)g.ntiles));
        const long long n = totals[s];
        Scratch scr(c);
        std::vector<long long> offs((size_t)g.ntiles);
        long long acc = 0;
        for (int t = 0; t < g.ntiles; ++t) {
            offs[t] = acc;
            acc += counts[s][t];
        }
        long long *doffs = nullptr;
        float *arr[9] = {};
        uint64_t *ids = nullptr;
        bool ok = scr.get((void **)&doffs, sizeof(long long) * offs.size());
        for (int k = 0; ok && k < 9; ++k) {
            if ((k == 7 && !d.zq) || (k == 8 && !d.tau)) continue;
            ok = scr.get((void **)&arr[k], sizeof(float) * (size_t)std::max(n, 1LL));
        }
        if (ok) ok = scr.get((void **)&ids, sizeof(uint64_t) * (size_t)std::max(n, 1LL));
        if (!ok) return set_error(HYB_ENOMEM, "staging memory for the particle checkpoint");
        HYB_CUDA_TRY(cudaMemcpyAsync(doffs, offs.data(), sizeof(long long) * offs.size(), cudaMemcpyHostToDevice,
                                     c->stream));
        launch_tiles_to_arrays(g, d, doffs, arr[0], arr[1], arr[2], arr[3], arr[4], arr[5], arr[6], arr[7], arr[8],
                               ids, c->stream);
        HYB_CUDA_TRY(cudaGetLastError());
        for (int k = 0; k < 9; ++k)
            if (arr[k]) HYB_CUDA_TRY(put_dev(arr[k], sizeof(float) * (size_t)n));
        HYB_CUDA_TRY(put_dev(ids, sizeof(uint64_t) * (size_t)n));
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    for (const FluidDev &f : c->fluids) {
        FluidHeader fh;
        std::memset(&fh, 0, sizeof(fh));
        fh.q = f.q;
        fh.m = f.m_d;
        HYB_CUDA_TRY(cudaMemcpyAsync(&fh.clamped, f.clamped, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                     c->stream));
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        put_host(&fh, sizeof(fh));
        const float *arrs[4] = {f.n, f.ux, f.uy, f.uz};
        for (const float *a : arrs) HYB_CUDA_TRY(put_dev(a, sizeof(float) * N));
    }
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (off != bytes) return set_error(HYB_ECUDA, "internal: state size mismatch");
    return HYB_OK;
}

hyb_status hyb_set_state(hyb_ctx *c, const void *buf, size_t size) {
    if (!c || !buf) return set_error(HYB_EINVAL, "null argument");
    const GridDev &g = c->g;
    const size_t N = (size_t)g.N;
    const char *in = static_cast<const char *>(buf);
    if (size < sizeof(StateHeader)) return set_error(HYB_EINVAL, "state image too short");
    StateHeader h;
    std::memcpy(&h, in, sizeof(h));
    if (std::memcmp(h.magic, STATE_MAGIC, 8) != 0 || h.version != STATE_VERSION || h.header_bytes != sizeof(h))
        return set_error(HYB_EINVAL, "not a state image of this library version");
    if (h.total_bytes != size) return set_error(HYB_EINVAL, "state image size does not match its header");
    bool same = h.T == g.T && h.order == g.order && h.seed == g.seed && h.dt == g.dt_d &&
                h.mur_plane == c->mur_plane;
    for (int a = 0; a < 3; ++a) same = same && h.n[a] == g.n[a] && h.bc[a] == g.bc[a] && h.d[a] == g.dd[a];
    if (!same) return set_error(HYB_EINVAL, "state image of a different grid, time step or seed");
    if (h.n_species != (int)c->sp.size() || h.n_fluids != (int)c->fluids.size())
        return set_error(HYB_EINVAL, "state image with other species or fluids than the context");
    // validate every section header before touching the device
    {
        size_t off = pad8(sizeof(StateHeader)) + 3 * 3 * pad8(sizeof(float) * N) +
                     pad8(sizeof(float) * 24 * (size_t)c->mur_plane) + pad8(sizeof(float) * N) + 2 * pad8(N);
        for (size_t s = 0; s < c->sp.size(); ++s) {
            if (off + sizeof(SpeciesHeader) > size) return set_error(HYB_EINVAL, "state image truncated");
            SpeciesHeader sh;
            std::memcpy(&sh, in + off, sizeof(sh));
            const SpDev &d = c->sp[s].dev;
            if (sh.q != c->sp[s].q || sh.m != c->sp[s].m || sh.kind != d.kind || sh.zmax != d.zmax ||
                sh.has_zq != (d.zq ? 1 : 0) || sh.has_tau != (d.tau ? 1 : 0) || sh.n < 0 || sh.cap <= 0)
                return set_error(HYB_EINVAL, "state image species " + std::to_string(s) + " differs from the context's");
            off += species_bytes(c->sp[s], sh.n, g.ntiles);
        }
        for (size_t f = 0; f < c->fluids.size(); ++f) {
            if (off + sizeof(FluidHeader) > size) return set_error(HYB_EINVAL, "state image truncated");
            FluidHeader fh;
            std::memcpy(&fh, in + off, sizeof(fh));
            if (fh.q != (double)c->fluids[f].q || fh.m != c->fluids[f].m_d)
                return set_error(HYB_EINVAL, "state image fluid " + std::to_string(f) + " differs from the context's");
            off += pad8(sizeof(FluidHeader)) + 4 * pad8(sizeof(float) * N);
        }
        if (off != size) return set_error(HYB_EINVAL, "state image size does not match its sections");
    }
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    size_t off = pad8(sizeof(StateHeader));
    auto get_dev = [&](void *dst, size_t b) -> cudaError_t {
        const cudaError_t e = cudaMemcpyAsync(dst, in + off, b, cudaMemcpyHostToDevice, c->stream);
        off += pad8(b);
        return e;
    };
    float *fields[3] = {c->E, c->B, c->J};
    for (float *f : fields)
        for (int q = 0; q < 3; ++q) HYB_CUDA_TRY(get_dev(f + q * N, sizeof(float) * N));
    HYB_CUDA_TRY(get_dev(c->mur_old, sizeof(float) * 24 * (size_t)c->mur_plane));
    HYB_CUDA_TRY(get_dev(c->rho_bg, sizeof(float) * N));
    HYB_CUDA_TRY(get_dev(c->mask, N));
    HYB_CUDA_TRY(get_dev(c->mask_prev, N));
    int status = 0;
    for (size_t s = 0; s < c->sp.size(); ++s) {
        Species &sp = c->sp[s];
        SpeciesHeader sh;
        std::memcpy(&sh, in + off, sizeof(sh));
        off += pad8(sizeof(sh));
        if (sh.cap != sp.cap) {
            // the saved tile capacity, so that later growth happens at the same fill
            HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
            SpDev ns = sp.dev;
            if (alloc_slots(c, ns, sh.cap, sp.dev.zq != nullptr, sp.dev.tau != nullptr) != HYB_OK)
                return set_error(HYB_ENOMEM, "slots for the restored tile capacity");
            free_slots(c, sp.dev);
            sp.dev = ns;
            sp.cap = sh.cap;
            sp.mig_cap = ns.mig_cap;
        }
        SpDev &d = sp.dev;
        HYB_CUDA_TRY(get_dev(d.tal_e, sizeof(double) * NTALLY * (size_t)g.ntiles));
        HYB_CUDA_TRY(get_dev(d.tal_n, sizeof(unsigned long long) * NTALLY * (size_t)g.ntiles));
        HYB_CUDA_TRY(cudaMemsetAsync(d.count, 0, sizeof(int) * g.ntiles, c->stream));
        HYB_CUDA_TRY(cudaMemsetAsync(d.hole_count, 0, sizeof(int) * g.ntiles, c->stream));
        HYB_CUDA_TRY(cudaMemsetAsync(d.hole_used, 0, sizeof(int) * g.ntiles, c->stream));
        const long long n = sh.n;
        Scratch scr(c);
        float *arr[9] = {};
        uint64_t *ids = nullptr;
        bool ok = true;
        for (int k = 0; ok && k < 9; ++k) {
            if ((k == 7 && !d.zq) || (k == 8 && !d.tau)) continue;
            ok = scr.get((void **)&arr[k], sizeof(float) * (size_t)std::max(n, 1LL));
        }
        if (ok) ok = scr.get((void **)&ids, sizeof(uint64_t) * (size_t)std::max(n, 1LL));
        if (!ok) return set_error(HYB_ENOMEM, "staging memory for the particle restore");
        for (int k = 0; k < 9; ++k)
            if (arr[k]) HYB_CUDA_TRY(get_dev(arr[k], sizeof(float) * (size_t)n));
        HYB_CUDA_TRY(get_dev(ids, sizeof(uint64_t) * (size_t)n));
        launch_bin_particles(g, d, n, arr[0], arr[1], arr[2], arr[3], arr[4], arr[5], arr[6], arr[7], ids, arr[8],
                             c->status, c->stream);
        HYB_CUDA_TRY(cudaGetLastError());
        HYB_CUDA_TRY(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (status) return set_error(HYB_EOVERFLOW, "restored particles do not fit their tiles");
    }
    for (FluidDev &f : c->fluids) {
        FluidHeader fh;
        std::memcpy(&fh, in + off, sizeof(fh));
        off += pad8(sizeof(fh));
        HYB_CUDA_TRY(cudaMemcpyAsync(f.clamped, &fh.clamped, sizeof(unsigned long long), cudaMemcpyHostToDevice,
                                     c->stream));
        float *arrs[4] = {f.n, f.ux, f.uy, f.uz};
        for (float *a : arrs) HYB_CUDA_TRY(get_dev(a, sizeof(float) * N));
        HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    // counters, flags and the species table
    c->step = h.step;
    c->epoch = h.epoch;
    c->regime = h.regime;
    // the fluid kernels cover every plane again until the next classification (after a step)
    c->fluid_fresh_step = h.step;
    if (clear_fluid_range(c, c->stream) != HYB_OK) return set_error(HYB_ECUDA, "fluid range reset");
    if (c->fluids_idle != (h.fluids_idle != 0)) c->fluids_idle = h.fluids_idle != 0;
    HYB_CUDA_TRY(cudaMemcpyAsync(c->step_dev, &h.step, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    HYB_CUDA_TRY(cudaMemcpyAsync(c->status, &h.status, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    HYB_CUDA_TRY(cudaMemsetAsync(c->fill_flags, 0, sizeof(int), c->stream));
    const SpSet all = species_set(c);
    if (all.n > 0)
        HYB_CUDA_TRY(cudaMemcpyAsync(c->sp_dev, all.s, sizeof(SpDev) * all.n, cudaMemcpyHostToDevice, c->stream));
    HYB_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->error_latched = h.status != 0;
    c->fill_pending = false;
    c->steps_since_copy = 0;
    c->graph_valid = false;
    return HYB_OK;
}

}  // extern "C"
