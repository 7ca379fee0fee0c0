// C ABI of the GB300 PC-LSQR library: handle creation (copy, layout and
// validation of the Gaia system), the two products, the preconditioner and
// the whole PC-LSQR solve.  No torch types cross this boundary.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "gsr_internal.cuh"

namespace gsr {
cudaError_t enqueue_precondition(const gsr_handle_t *h, double *p, cudaStream_t st);
int aprod2_grid(const gsr_handle_t *h);
int aprod2_fused_grid(const gsr_handle_t *h);
}  // namespace gsr

using namespace gsr;

static thread_local char g_last_error[256] = "";

static int cuda_fail(cudaError_t e, const char *what)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return GSR_ERR_CUDA;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess)                                       \
            return e_ == cudaErrorMemoryAllocation                   \
                       ? (snprintf(g_last_error, sizeof g_last_error, \
                                   "%s: out of memory", #call),      \
                          cudaGetLastError(), GSR_ERR_OOM)           \
                       : cuda_fail(e_, #call);                       \
    } while (0)

extern "C" const char *gsr_last_error(void) { return g_last_error; }

extern "C" const char *gsr_strerror(int code)
{
    switch (code) {
    case GSR_OK: return "success";
    case GSR_ERR_ARG: return "invalid argument";
    case GSR_ERR_INDEX: return "matrix structure out of range";
    case GSR_ERR_OOM: return "out of memory";
    case GSR_ERR_CUDA: return "CUDA runtime error";
    case GSR_ERR_NONFINITE: return "non-finite value";
    case GSR_ERR_UNSUPPORTED: return "unsupported configuration";
    case GSR_ERR_TIMEOUT: return "a bounded device wait expired";
    default: return "unknown error";
    }
}

extern "C" void gsr_config_default(gsr_config *c)
{
    if (!c)
        return;
    memset(c, 0, sizeof *c);
    c->precision = GSR_PREC_FP64;
    c->conlim = 1e8;
    c->lanes_per_star = 0;
    c->validate = 1;
}

// instrument index j (0..5) of a packed row record
static inline uint32_t instr_of(const uint4 &r, int j)
{
    const uint32_t w = j < 2 ? r.y : (j < 4 ? r.z : r.w);
    return (j & 1) ? (w >> 16) : (w & 0xffffu);
}

static bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static int dalloc(gsr_handle_t *h, T **p, int64_t count)
{
    const size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        snprintf(g_last_error, sizeof g_last_error, "cudaMalloc(%zu bytes): %s", bytes,
                 cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GSR_ERR_OOM : GSR_ERR_CUDA;
    }
    h->device_bytes += (int64_t)bytes;
    return GSR_OK;
}

#define TRY(x)                \
    do {                      \
        int rc_ = (x);        \
        if (rc_ != GSR_OK)    \
            return rc_;       \
    } while (0)

static void release(gsr_handle_t *h)
{
    if (!h)
        return;
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    if (h->solve_exec)
        cudaGraphExecDestroy(h->solve_exec);
    if (h->cg_exec)
        cudaGraphExecDestroy(h->cg_exec);
    if (h->cg64_exec)
        cudaGraphExecDestroy(h->cg64_exec);
    if (h->b_exec)
        cudaGraphExecDestroy(h->b_exec);
    if (h->h_bs)
        cudaFreeHost(h->h_bs);
    if (h->h_bargs)
        cudaFreeHost(h->h_bargs);
    if (h->h_bnorms)
        cudaFreeHost(h->h_bnorms);
    if (h->h_cg)
        cudaFreeHost(h->h_cg);
    if (h->h_cgargs)
        cudaFreeHost(h->h_cgargs);
    if (h->h_onorm)
        cudaFreeHost(h->h_onorm);
    if (h->cap_stream)
        cudaStreamDestroy(h->cap_stream);
    void *dev[] = {h->d_star_ptr, h->d_rec, h->d_val, h->d_tile_star, h->d_sdelta, h->d_sorder, h->d_tval, h->d_perm,
                   h->d_seg, h->d_attS, h->d_irep, h->d_p, h->d_u, h->d_v, h->d_w, h->d_z,
                   h->d_var, h->d_q, h->d_vp, h->d_vt, h->d_bstage, h->d_xstage, h->d_sestage,
                   h->d_ystage, h->d_state, h->d_args, h->d_partial, h->d_counter, h->d_err,
                   h->d_val32, h->d_tval32, h->d_x32, h->d_xatt4, h->d_q32, h->d_c, h->d_s, h->d_d, h->d_t,
                   h->d_zc, h->d_xm, h->d_r, h->d_xneg, h->d_onorm, h->d_cg, h->d_cgargs,
                   h->d_xp64, h->d_q64, h->d_iseg, h->d_cseg, h->d_cseg32, h->d_irow, h->d_ival32, h->d_ival, h->d_ipart, h->d_gpart, h->d_a2ctr, h->d_bX32, h->d_bQ32,
                   h->d_bC, h->d_bS_, h->d_bD, h->d_bZ, h->d_bT, h->d_bS, h->d_bXcm,
                   h->d_bCcm, h->d_bB, h->d_bnorms, h->d_bpartial, h->d_bcounter, h->d_bs,
                   h->d_bipart,
                   h->d_bargs};
    for (void *p : dev)
        if (p)
            cudaFree(p);
    if (h->h_state)
        cudaFreeHost(h->h_state);
    if (h->h_args)
        cudaFreeHost(h->h_args);
    cudaGetLastError();
    if (cur >= 0)
        cudaSetDevice(cur);
    delete h;
}

// Instrument-sorted copy of the instrumental nonzeros: a stable counting
// sort of the 6 m entries (row, slot) by instrument on the host, so the
// entries of every instrument keep ascending row order and their sums a
// fixed order; the FP64 values are then gathered on the device.  The
// entries of each instrument are cut at row windows of R rows (a unit of
// the instrumental sums is one instrument in one window): units are taken
// window by window, so the y entries they gather stay within R rows, which
// L2 holds also when the whole of y does not fit; R also bounds a unit to
// about 4096 entries.
static int build_instr_sorted(gsr_handle_t *h, cudaStream_t st)
{
    SysView &A = h->sys;
    const int64_t m = A.m, I = A.I, E = kNInstr * m;
    std::vector<uint4> rec((size_t)m);
    CK(cudaMemcpy(rec.data(), h->d_rec, m * sizeof(uint4), cudaMemcpyDeviceToHost));
    std::vector<uint32_t> seg((size_t)I + 1, 0);
    for (int64_t i = 0; i < m; i++)
        for (int j = 0; j < kNInstr; j++)
            seg[instr_of(rec[i], j) + 1]++;
    for (int64_t f = 0; f < I; f++)
        seg[f + 1] += seg[f];
    std::vector<uint32_t> pos(seg.begin(), seg.end() - 1), irow((size_t)E), code((size_t)E);
    for (int64_t i = 0; i < m; i++)
        for (int j = 0; j < kNInstr; j++) {
            const uint32_t p = pos[instr_of(rec[i], j)]++;
            irow[p] = (uint32_t)i;
            code[p] = (uint32_t)(kNInstr * i + j);
        }
    std::vector<uint4>().swap(rec);
    TRY(dalloc(h, &h->d_iseg, I + 1));
    TRY(dalloc(h, &h->d_irow, E));
    TRY(dalloc(h, &h->d_ival, E));
    CK(cudaMemcpy(h->d_iseg, seg.data(), (I + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->d_irow, irow.data(), E * sizeof(uint32_t), cudaMemcpyHostToDevice));
    uint32_t *d_code = nullptr;
    if (cudaMalloc(&d_code, E * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return GSR_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(d_code, code.data(), E * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_gather_instr64(h, d_code, h->d_ival, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(d_code);
    if (e != cudaSuccess)
        return cuda_fail(e, "instrument-sorted layout");
    // row windows: R = 4096 I / 6 rows (about 4096 entries per instrument and
    // window), at most 4 Mi rows (32 MB of FP64 y), at least 64 Ki rows
    int64_t R = 4096 * I / kNInstr;
    if (R > ((int64_t)1 << 22))
        R = (int64_t)1 << 22;
    if (R < ((int64_t)1 << 16))
        R = (int64_t)1 << 16;
    const int64_t nq = (m + R - 1) / R;
    std::vector<uint32_t> cseg((size_t)((nq + 1) * I));
    for (int64_t f = 0; f < I; f++) {
        uint32_t e = seg[f];
        for (int64_t q = 0; q < nq; q++) {
            cseg[q * I + f] = e;
            const int64_t rend = (q + 1) * R;  // entries of window q: rows < rend
            while (e < seg[f + 1] && (int64_t)irow[e] < rend)
                e++;
        }
        cseg[nq * I + f] = seg[f + 1];
    }
    TRY(dalloc(h, &h->d_cseg, (nq + 1) * I));
    CK(cudaMemcpy(h->d_cseg, cseg.data(), (nq + 1) * I * sizeof(uint32_t), cudaMemcpyHostToDevice));
    h->isplit = (int)nq;
    int64_t nparts = nq;
    if (h->cfg.precision == GSR_PREC_MIXED) {
        // binary32 units: windows of 32 MB of binary32 y (8 Mi rows), each
        // instrument's window cut by count into ks32 pieces of <= 4096 entries
        const int64_t R32 = (int64_t)1 << 23;
        const int64_t nq32 = (m + R32 - 1) / R32;
        const int64_t per = kNInstr * (R32 < m ? R32 : m) / I + 1;  // entries per window
        const int64_t ks32 = (per + 4095) / 4096;
        std::vector<uint32_t> c32((size_t)((nq32 + 1) * I));
        for (int64_t f = 0; f < I; f++) {
            uint32_t e = seg[f];
            for (int64_t q = 0; q < nq32; q++) {
                c32[q * I + f] = e;
                while (e < seg[f + 1] && (int64_t)irow[e] < (q + 1) * R32)
                    e++;
            }
            c32[nq32 * I + f] = seg[f + 1];
        }
        TRY(dalloc(h, &h->d_cseg32, (nq32 + 1) * I));
        CK(cudaMemcpy(h->d_cseg32, c32.data(), (nq32 + 1) * I * sizeof(uint32_t),
                      cudaMemcpyHostToDevice));
        h->nq32 = (int)nq32;
        h->ks32 = (int)ks32;
        if (nq32 * ks32 > nparts)
            nparts = nq32 * ks32;
    }
    TRY(dalloc(h, &h->d_ipart, nparts * I));
    CK(cudaMemset(h->d_ipart, 0, (size_t)nparts * I * sizeof(double)));
    const int64_t units_blocks = (I * h->isplit + kThreads / 32 - 1) / (kThreads / 32);
    const int64_t cap = (int64_t)h->nsm * 16;
    h->grid_ins = (int)(units_blocks < cap ? units_blocks : cap);
    return GSR_OK;
}

// binary32 copies of the value planes and of the offset-sorted attitude
// values, the mixed-precision workspace and the inner CG graph
static int create_mixed(gsr_handle_t *h, cudaStream_t st)
{
    SysView &A = h->sys;
    const int64_t m = A.m, n = A.n, mp = A.mp;
    TRY(dalloc(h, &h->d_val32, kNPar * mp));
    TRY(dalloc(h, &h->d_tval32, (int64_t)kNAtt * mp));
    TRY(dalloc(h, &h->d_ival32, kNInstr * m));
    TRY(dalloc(h, &h->d_x32, n));
    TRY(dalloc(h, &h->d_xatt4, 3 * A.D * 4));
    CK(cudaMemset(h->d_xatt4, 0, 3 * A.D * 4 * sizeof(float)));
    TRY(dalloc(h, &h->d_q32, m));
    CK(launch_to_f32(h, h->d_val, h->d_val32, kNPar * mp, st));
    CK(launch_to_f32(h, h->d_tval, h->d_tval32, kNAtt * mp, st));
    A.val32 = h->d_val32;
    A.tval32 = h->d_tval32;
    CK(launch_to_f32(h, h->d_ival, h->d_ival32, kNInstr * m, st));
    // ||A diag(p)||_F^2 = number of nonempty columns (column sums of squares > 0)
    CK(cudaMemsetAsync(h->d_s, 0, n * sizeof(double), st));
    CK(launch_aprod2(h, nullptr, h->d_s, kA2Squares, st));
    CK(launch_count_pos(h, h->d_s, h->d_onorm, st));
    CK(cudaMemcpyAsync(h->h_onorm, h->d_onorm, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    h->n_nonempty = h->h_onorm[0];
    h->grid_rows32 = aprod1_f32_grid(h);
    h->grid_rows2_32 = aprod2_f32_grid(h);
    h->grid_fused32 = aprod2_f32_fused_grid(h);
    if (h->grid_rows32 <= 0 || h->grid_rows2_32 <= 0 || h->grid_fused32 <= 0)
        return cuda_fail(cudaGetLastError(), "mixed occupancy");
    cudaError_t e = build_cg_graph(h);
    if (e != cudaSuccess)
        return cuda_fail(e, "build_cg_graph");
    return GSR_OK;
}

static int create_impl(gsr_handle_t *h, const gsr_dims *d, const uint32_t *star_ptr,
                       const uint32_t *attoff, const uint16_t *instr, const double *values)
{
    const int64_t S = d->n_stars, D = d->n_dfa, I = d->n_instr, m = d->n_rows;
    const int64_t n = kNAstro * S + 3 * D + I + 1;
    const int64_t mp = (m + 31) / 32 * 32;
    cudaDeviceProp prop;
    CK(cudaGetDevice(&h->device));
    CK(cudaGetDeviceProperties(&prop, h->device));
    h->nsm = prop.multiProcessorCount;

    SysView &A = h->sys;
    A.S = S; A.D = D; A.I = I; A.m = m; A.n = n; A.mp = mp;
    A.att0 = kNAstro * S;
    A.ins0 = A.att0 + 3 * D;
    A.glb0 = A.ins0 + I;
    A.nseg = D - 3;
    const int64_t ntiles = (m + 31) / 32;

    TRY(dalloc(h, &h->d_star_ptr, S + 1));
    // records and star deltas padded to whole 32-row tiles (zero), so a tile
    // can be staged by one bulk copy
    TRY(dalloc(h, &h->d_rec, mp));
    TRY(dalloc(h, &h->d_val, kNPar * mp));
    TRY(dalloc(h, &h->d_tile_star, ntiles));
    TRY(dalloc(h, &h->d_sdelta, mp));
    TRY(dalloc(h, &h->d_sorder, S));
    TRY(dalloc(h, &h->d_tval, (int64_t)kNAtt * mp));
    TRY(dalloc(h, &h->d_perm, m));
    TRY(dalloc(h, &h->d_seg, A.nseg + 1));
    TRY(dalloc(h, &h->d_attS, A.nseg * kNAtt));
    TRY(dalloc(h, &h->d_p, n));
    TRY(dalloc(h, &h->d_u, m));
    TRY(dalloc(h, &h->d_v, n));
    TRY(dalloc(h, &h->d_w, n));
    TRY(dalloc(h, &h->d_z, n));
    TRY(dalloc(h, &h->d_var, n));
    TRY(dalloc(h, &h->d_q, n));
    TRY(dalloc(h, &h->d_vp, n));
    TRY(dalloc(h, &h->d_state, 1));
    TRY(dalloc(h, &h->d_args, 1));
    TRY(dalloc(h, &h->d_partial, (int64_t)kRedCount * kPartialsPerKind));
    TRY(dalloc(h, &h->d_counter, kRedCount));
    TRY(dalloc(h, &h->d_err, 1));
    TRY(dalloc(h, &h->d_kerr, 1));
    CK(cudaMemset(h->d_counter, 0, kRedCount * sizeof(unsigned)));
    CK(cudaMemset(h->d_err, 0, sizeof(int)));
    CK(cudaMemset(h->d_kerr, 0, sizeof(int)));
    CK(cudaMemset(h->d_rec, 0, (size_t)mp * sizeof(uint4)));
    CK(cudaMemset(h->d_sdelta, 0, (size_t)mp * sizeof(uint16_t)));
    CK(cudaMemset(h->d_val, 0, (size_t)kNPar * mp * sizeof(double)));
    CK(cudaMallocHost((void **)&h->h_state, sizeof(SolveState)));
    CK(cudaMallocHost((void **)&h->h_args, sizeof(SolveArgs)));
    A.star_ptr = h->d_star_ptr;
    A.rec = h->d_rec;
    A.val = h->d_val;
    A.tile_star = h->d_tile_star;
    A.sdelta = h->d_sdelta;
    A.sorder = h->d_sorder;
    A.tval = h->d_tval;
    A.perm = h->d_perm;
    A.seg = h->d_seg;

    CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t st = h->cap_stream;

    // star_ptr: host arrays are checked here; all of it again on the device
    if (!on_device(star_ptr) && (star_ptr[0] != 0 || (int64_t)star_ptr[S] != m))
        return GSR_ERR_INDEX;
    CK(cudaMemcpyAsync(h->d_star_ptr, star_ptr, (S + 1) * sizeof(uint32_t), cudaMemcpyDefault, st));

    // index records and value planes, staged in chunks of rows
    const int64_t chunk = 1 << 20;
    const bool rec_dev = on_device(attoff) && on_device(instr);
    const bool val_dev = on_device(values);
    uint32_t *s_att = nullptr;
    uint16_t *s_ins = nullptr;
    double *s_val = nullptr;
    int rc = GSR_OK;
    if (!rec_dev) {
        if (cudaMalloc(&s_att, chunk * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&s_ins, chunk * kNInstr * sizeof(uint16_t)) != cudaSuccess)
            rc = GSR_ERR_OOM;
    }
    if (rc == GSR_OK && !val_dev && cudaMalloc(&s_val, chunk * kNPar * sizeof(double)) != cudaSuccess)
        rc = GSR_ERR_OOM;
    for (int64_t r0 = 0; rc == GSR_OK && r0 < m; r0 += chunk) {
        const int64_t nr = (m - r0 < chunk) ? m - r0 : chunk;
        cudaError_t e = cudaSuccess;
        if (rec_dev) {
            e = launch_pack_rec(h, attoff + r0, instr + kNInstr * r0, r0, nr, st);
        } else {
            e = cudaMemcpyAsync(s_att, attoff + r0, nr * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s_ins, instr + kNInstr * r0, nr * kNInstr * sizeof(uint16_t),
                                    cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = launch_pack_rec(h, s_att, s_ins, r0, nr, st);
        }
        if (e == cudaSuccess) {
            if (val_dev) {
                e = launch_planes(h, values + kNPar * r0, r0, nr, st);
            } else {
                e = cudaMemcpyAsync(s_val, values + kNPar * r0, nr * kNPar * sizeof(double),
                                    cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess)
                    e = launch_planes(h, s_val, r0, nr, st);
            }
        }
        if (e == cudaSuccess && !(rec_dev && val_dev))
            e = cudaStreamSynchronize(st);  // staging buffers are reused
        if (e != cudaSuccess)
            rc = cuda_fail(e, "layout");
    }
    if (s_att) cudaFree(s_att);
    if (s_ins) cudaFree(s_ins);
    if (s_val) cudaFree(s_val);
    if (rc != GSR_OK)
        return rc;

    // validation of the structure (always) and of the values (cfg.validate)
    CK(launch_validate(h, st));
    int err = 0;
    CK(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err & 7)
        return GSR_ERR_INDEX;
    if (err & 8)
        return GSR_ERR_NONFINITE;

    // stars in decreasing row count (stable): the star groups of aprod 2
    {
        std::vector<uint32_t> sp((size_t)S + 1), order((size_t)S);
        CK(cudaMemcpy(sp.data(), h->d_star_ptr, (S + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        for (int64_t s = 0; s < S; s++)
            order[s] = (uint32_t)s;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
            return sp[a + 1] - sp[a] > sp[b + 1] - sp[b];
        });
        CK(cudaMemcpy(h->d_sorder, order.data(), S * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }

    // attitude copy sorted by offset: a stable counting sort on the host
    // (row order kept inside every offset, so the sums have a fixed order)
    {
        std::vector<uint32_t> att_host;
        const uint32_t *ao = attoff;
        if (on_device(attoff)) {
            att_host.resize((size_t)m);
            CK(cudaMemcpy(att_host.data(), attoff, m * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            ao = att_host.data();
        }
        std::vector<uint32_t> seg((size_t)A.nseg + 1, 0), perm((size_t)m);
        for (int64_t i = 0; i < m; i++) {
            if ((int64_t)ao[i] >= A.nseg)
                return GSR_ERR_INDEX;
            seg[ao[i] + 1]++;
        }
        for (int64_t o = 0; o < A.nseg; o++)
            seg[o + 1] += seg[o];
        std::vector<uint32_t> pos(seg.begin(), seg.end() - 1);
        for (int64_t i = 0; i < m; i++)
            perm[pos[ao[i]]++] = (uint32_t)i;
        CK(cudaMemcpy(h->d_perm, perm.data(), m * sizeof(uint32_t), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->d_seg, seg.data(), (A.nseg + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    CK(launch_gather_att(h, st));
    CK(launch_tile_star(h, st));
    CK(cudaStreamSynchronize(st));

    // instrumental part of aprod 2 and its layout
    h->ipath = instr_path(h->cfg, I);
    if (h->ipath == kIpSorted || h->cfg.precision == GSR_PREC_MIXED)
        TRY(build_instr_sorted(h, st));

    // launch geometry
    // measured at the medium size: 8 lanes per star with shared-memory
    // instrument sums or the sorted pass, 32 with replicas
    h->lanes = h->cfg.lanes_per_star ? h->cfg.lanes_per_star : (h->ipath == kIpReplicas ? 32 : 8);
    // aprod 1 staged by the bulk-copy engine wherever it applies (measured
    // faster in the solve on the medium workload: 0.305 against 0.328 ms)
    CK(aprod1_tma_prepare(h));
    h->a1_tma = h->a1_tma_avail;
    h->grid_rows = aprod1_grid(h);
    if (h->grid_rows <= 0)
        return cuda_fail(cudaGetLastError(), "aprod1 occupancy");
    h->grid_att = h->nsm * 8;
    // vector kernels: two blocks per SM (each thread takes several entries,
    // so the per-block reduction epilogue stays a small share of the work)
    int64_t gv = (n + kThreads - 1) / kThreads;
    if (gv > (int64_t)h->nsm * 2) gv = (int64_t)h->nsm * 2;
    if (gv > kMaxPartials) gv = kMaxPartials;
    h->grid_vec = (int)(gv < 1 ? 1 : gv);
    h->grid_lsqr_vec = lsqr_vec_grid(h);
    if (h->grid_lsqr_vec <= 0)
        return cuda_fail(cudaGetLastError(), "vector pass occupancy");
    if (h->ipath == kIpReplicas || (h->cfg.precision == GSR_PREC_MIXED && !instr_in_smem(h))) {
        h->nrep = h->nsm;
        TRY(dalloc(h, &h->d_irep, (int64_t)h->nrep * I));
        CK(cudaMemset(h->d_irep, 0, (size_t)h->nrep * I * sizeof(double)));
    }
    h->grid_rows2 = aprod2_grid(h);
    if (h->grid_rows2 <= 0)
        return cuda_fail(cudaGetLastError(), "aprod2 occupancy");
    int ngp = h->grid_rows2;
    if (h->ipath == kIpSorted) {
        h->grid_fused = aprod2_fused_grid(h);
        if (h->grid_fused <= 0)
            return cuda_fail(cudaGetLastError(), "fused aprod2 occupancy");
        // star units of the FP64 and of the binary32 (4 stars each) launches
        int64_t nsu = (h->sys.S + 32 / h->lanes - 1) / (32 / h->lanes);
        const int64_t nsu32 = (h->sys.S + 3) / 4;
        if (nsu32 > nsu)
            nsu = nsu32;
        if (nsu > ((int64_t)1 << 30) || a2_queue(h, h->lanes).total >= ((int64_t)1 << 32))
            h->a2_fused = 0;  // bounded partials buffer; 32-bit unit indices
        else if (nsu > ngp)
            ngp = (int)nsu;
        TRY(dalloc(h, &h->d_a2ctr, 1));
        CK(cudaMemset(h->d_a2ctr, 0, sizeof(unsigned long long)));
    } else {
        h->a2_fused = 0;
    }
    TRY(dalloc(h, &h->d_gpart, ngp));

    // scratch of gsr_aprod1_norm_noalloc: resolved here, where allocating is
    // allowed, so that entry point never loads a module or allocates
    TRY(noalloc_prepare(h->device));
    cudaError_t e = build_solve_graph(h);
    if (e != cudaSuccess)
        return cuda_fail(e, "build_solve_graph");
    // conjugate-gradient workspace (normal-equation solves of the adjoint and
    // of the mixed-precision refinement)
    TRY(dalloc(h, &h->d_c, n));
    TRY(dalloc(h, &h->d_s, n));
    TRY(dalloc(h, &h->d_d, n));
    TRY(dalloc(h, &h->d_t, n));
    TRY(dalloc(h, &h->d_zc, n));
    TRY(dalloc(h, &h->d_xm, n));
    TRY(dalloc(h, &h->d_xp64, n));
    TRY(dalloc(h, &h->d_xneg, n));
    TRY(dalloc(h, &h->d_r, m));
    TRY(dalloc(h, &h->d_q64, m));
    TRY(dalloc(h, &h->d_onorm, 4));
    TRY(dalloc(h, &h->d_cg, 1));
    TRY(dalloc(h, &h->d_cgargs, 1));
    CK(cudaMallocHost((void **)&h->h_cg, sizeof(CgState)));
    CK(cudaMallocHost((void **)&h->h_cgargs, sizeof(CgArgs)));
    CK(cudaMallocHost((void **)&h->h_onorm, 4 * sizeof(double)));
    e = build_cg64_graph(h);
    if (e != cudaSuccess)
        return cuda_fail(e, "build_cg64_graph");
    if (h->cfg.precision == GSR_PREC_MIXED)
        return create_mixed(h, st);
    return GSR_OK;
}

extern "C" int gsr_create(void **out, const gsr_dims *d, const uint32_t *star_ptr,
                          const uint32_t *attoff, const uint16_t *instr, const double *values,
                          const gsr_config *cfg)
{
    if (!out || !d || !star_ptr || !attoff || !instr || !values)
        return GSR_ERR_ARG;
    if (d->n_stars < 1 || d->n_dfa < 4 || d->n_instr < kNInstr || d->n_instr > 65536 ||
        d->n_rows < 1 || d->n_rows >= ((int64_t)1 << 32) - 32)
        return GSR_ERR_ARG;
    gsr_config c;
    if (cfg)
        c = *cfg;
    else
        gsr_config_default(&c);
    if (c.precision != GSR_PREC_FP64 && c.precision != GSR_PREC_MIXED)
        return GSR_ERR_UNSUPPORTED;
    if (c.lanes_per_star != 0 && c.lanes_per_star != 4 && c.lanes_per_star != 8 &&
        c.lanes_per_star != 16 && c.lanes_per_star != 32)
        return GSR_ERR_ARG;
    if (!(c.conlim >= 0.0))
        return GSR_ERR_ARG;
    if (c.instr_mode < GSR_INSTR_AUTO || c.instr_mode > GSR_INSTR_SORTED)
        return GSR_ERR_ARG;
    if (c.instr_mode == GSR_INSTR_SMEM && d->n_instr > 6144)
        return GSR_ERR_UNSUPPORTED;
    if ((c.products < GSR_PRODUCTS_AUTO || c.products > GSR_PRODUCTS_SPLIT) &&
        (c.products & ~63) != GSR_PRODUCTS_MASK)
        return GSR_ERR_ARG;
    if ((c.products & ~63) == GSR_PRODUCTS_MASK) {
        const int r = c.products & 63;
        if ((r & GSR_SPLIT_APROD1_ASTRO) && !(r & GSR_SPLIT_APROD1))
            return GSR_ERR_ARG;
        if ((r & GSR_SPLIT_APROD2_ATT) && (r & GSR_SPLIT_APROD2_ATT2))
            return GSR_ERR_ARG;
        if ((r & (GSR_SPLIT_APROD2_ATT | GSR_SPLIT_APROD2_ATT2)) && (r & GSR_SPLIT_APROD2_STARS))
            return GSR_ERR_UNSUPPORTED;  // no kernel combines these forms
        if ((r & GSR_SPLIT_APROD2_ATT2) && (r & GSR_SPLIT_APROD2_INSTR))
            return GSR_ERR_UNSUPPORTED;
    }
    // an explicit request for aprod 1's split form needs the split
    // instrumental x in shared memory
    if (c.products != GSR_PRODUCTS_AUTO && (split_request(c) & GSR_SPLIT_APROD1) &&
        d->n_instr > 3072)
        return GSR_ERR_UNSUPPORTED;
    gsr_handle_t *h = new (std::nothrow) gsr_handle_t();
    if (!h)
        return GSR_ERR_OOM;
    h->cfg = c;
    int rc;
    try {  // the host-side sorts allocate O(m) vectors; no exception leaves the ABI
        rc = create_impl(h, d, star_ptr, attoff, instr, values);
    } catch (const std::bad_alloc &) {
        snprintf(g_last_error, sizeof g_last_error, "host allocation failed in gsr_create");
        rc = GSR_ERR_OOM;
    } catch (...) {
        snprintf(g_last_error, sizeof g_last_error, "unexpected host error in gsr_create");
        rc = GSR_ERR_CUDA;
    }
    if (rc != GSR_OK) {
        release(h);
        return rc;
    }
    *out = h;
    return GSR_OK;
}

extern "C" int gsr_destroy(void *hv)
{
    release((gsr_handle_t *)hv);
    return GSR_OK;
}

extern "C" int gsr_info(void *hv, int64_t *m, int64_t *n, int64_t *bytes)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h)
        return GSR_ERR_ARG;
    if (m) *m = h->sys.m;
    if (n) *n = h->sys.n;
    if (bytes) *bytes = h->device_bytes;
    return GSR_OK;
}

// a device buffer for a caller's pointer: the pointer itself, or a staging
// buffer owned by the handle
static int stage(gsr_handle_t *h, double **slot, int64_t count, const double *user,
                 double **dev, bool copy_in, cudaStream_t st)
{
    if (on_device(user)) {
        *dev = (double *)user;
        return GSR_OK;
    }
    if (!*slot)
        TRY(dalloc(h, slot, count));
    *dev = *slot;
    if (copy_in)
        CK(cudaMemcpyAsync(*slot, user, count * sizeof(double), cudaMemcpyHostToDevice, st));
    return GSR_OK;
}

// GSR_ERR_TIMEOUT when a bounded wait of a kernel on this handle expired
// since the last check (the flag is then cleared); synchronizes the stream
static int take_kernel_status(gsr_handle_t *h, cudaStream_t st)
{
    int kerr = 0;
    CK(cudaMemcpyAsync(&kerr, h->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (kerr == 0)
        return GSR_OK;
    CK(cudaMemsetAsync(h->d_kerr, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    snprintf(g_last_error, sizeof g_last_error, "%s",
             "a bounded wait of the staged aprod 1 expired: a bulk copy did not complete");
    return GSR_ERR_TIMEOUT;
}

extern "C" int gsr_kernel_status(void *hv, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h)
        return GSR_ERR_ARG;
    return take_kernel_status(h, (cudaStream_t)stream);
}

extern "C" int gsr_aprod1(void *hv, const double *x, double *y, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !x || !y)
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *dx, *dy;
    TRY(stage(h, &h->d_xstage, h->sys.n, x, &dx, true, st));
    TRY(stage(h, &h->d_ystage, h->sys.m, y, &dy, true, st));
    CK(launch_aprod1(h, dx, dy, 0, st));
    if (dy != y) {
        CK(cudaMemcpyAsync(y, dy, h->sys.m * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return GSR_OK;
}

extern "C" int gsr_aprod2(void *hv, const double *y, double *x, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !x || !y)
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *dx, *dy;
    TRY(stage(h, &h->d_ystage, h->sys.m, y, &dy, true, st));
    TRY(stage(h, &h->d_xstage, h->sys.n, x, &dx, true, st));
    CK(launch_aprod2(h, dy, dx, kA2Accumulate, st));
    if (dx != x) {
        CK(cudaMemcpyAsync(x, dx, h->sys.n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return GSR_OK;
}

extern "C" int gsr_precondition(void *hv, double *p, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !p)
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *dp;
    TRY(stage(h, &h->d_xstage, h->sys.n, p, &dp, false, st));
    CK(enqueue_precondition(h, dp, st));
    if (dp != p) {
        CK(cudaMemcpyAsync(p, dp, h->sys.n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return GSR_OK;
}

extern "C" int gsr_lsqr_solve(void *hv, const double *b, int itmax, double atol, double btol,
                              double *x, double *se, gsr_result *out, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !b || !x || itmax < 1 || !(atol >= 0.0) || !(btol >= 0.0))
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *db, *dx, *dse = nullptr;
    TRY(stage(h, &h->d_bstage, h->sys.m, b, &db, true, st));
    TRY(stage(h, &h->d_xstage, h->sys.n, x, &dx, false, st));
    if (se)
        TRY(stage(h, &h->d_sestage, h->sys.n, se, &dse, false, st));
    SolveArgs *a = h->h_args;
    a->b = db;
    a->x = dx;
    a->se = dse;
    a->itmax = itmax;
    a->force_itmax = h->cfg.force_itmax ? 1 : 0;
    a->atol = atol;
    a->btol = btol;
    a->ctol = (h->cfg.conlim > 0.0) ? 1.0 / h->cfg.conlim : 0.0;
    a->isdof = 1.0 / sqrt((h->sys.m > h->sys.n) ? (double)(h->sys.m - h->sys.n) : 1.0);
    CK(cudaMemcpyAsync(h->d_args, a, sizeof(SolveArgs), cudaMemcpyHostToDevice, st));
    if (h->cfg.eager) {
        // every launch from the host, the loop flag read back after each step
        CK(enqueue_prologue(h, st, 0, 0));
        CK(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int it = 0; it < itmax && !h->h_state->done; it++) {
            CK(enqueue_iteration(h, st, 0, 0));
            CK(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost,
                               st));
            CK(cudaStreamSynchronize(st));
        }
        CK(enqueue_epilogue(h, st));
    } else {
        CK(cudaGraphLaunch(h->solve_exec, st));
    }
    CK(cudaMemcpyAsync(h->h_state, h->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    if (dx != x)
        CK(cudaMemcpyAsync(x, dx, h->sys.n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (se && dse != se)
        CK(cudaMemcpyAsync(se, dse, h->sys.n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    TRY(take_kernel_status(h, st));
    const SolveState &s = *h->h_state;
    if (out) {
        out->istop = s.istop;
        out->itn = s.itn;
        out->rnorm = s.rnorm;
        out->arnorm = s.arnorm;
        out->anorm = s.anorm;
        out->acond = s.acond;
        out->xnorm = s.xnorm;
        out->bnorm = s.bnorm;
    }
    return s.nonfinite ? GSR_ERR_NONFINITE : GSR_OK;
}

extern "C" int gsr_time_iteration(void *hv, const double *b, int iters, double *ms3, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !b || !ms3 || iters < 1 || iters > 256)
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *db, *dx;
    TRY(stage(h, &h->d_bstage, h->sys.m, b, &db, true, st));
    if (!h->d_xstage)
        TRY(dalloc(h, &h->d_xstage, h->sys.n));
    dx = h->d_xstage;
    SolveArgs *a = h->h_args;
    a->b = db;
    a->x = dx;
    a->se = nullptr;
    a->itmax = iters;
    a->force_itmax = 1;
    a->atol = a->btol = 0.0;
    a->ctol = 0.0;
    a->isdof = 1.0 / sqrt((h->sys.m > h->sys.n) ? (double)(h->sys.m - h->sys.n) : 1.0);
    CK(cudaMemcpyAsync(h->d_args, a, sizeof(SolveArgs), cudaMemcpyHostToDevice, st));
    std::vector<cudaEvent_t> ev((size_t)3 * iters + 1, nullptr);
    int rc = GSR_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            rc = GSR_ERR_CUDA;
        }
    cudaError_t e = cudaSuccess;
    if (rc == GSR_OK)
        e = enqueue_prologue(h, st, 0, 0);
    if (rc == GSR_OK && e == cudaSuccess)
        e = cudaEventRecord(ev[0], st);
    for (int it = 0; rc == GSR_OK && e == cudaSuccess && it < iters; it++)
        e = enqueue_iteration_timed(h, st, ev.data() + 3 * it);
    if (rc == GSR_OK && e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    double sum[3] = {0.0, 0.0, 0.0};
    for (int it = 0; rc == GSR_OK && e == cudaSuccess && it < iters; it++)
        for (int k = 0; k < 3 && e == cudaSuccess; k++) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[3 * it + k], ev[3 * it + k + 1]);
            sum[k] += ms;
        }
    for (auto &x : ev)
        if (x)
            cudaEventDestroy(x);
    if (rc != GSR_OK)
        return rc;
    if (e != cudaSuccess)
        return cuda_fail(e, "gsr_time_iteration");
    for (int k = 0; k < 3; k++)
        ms3[k] = sum[k] / iters;
    return GSR_OK;
}

extern "C" int gsr_aprod1_f32(void *hv, const double *x, double *y, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !x || !y)
        return GSR_ERR_ARG;
    if (h->cfg.precision != GSR_PREC_MIXED)
        return GSR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    double *dx, *dy;
    TRY(stage(h, &h->d_xstage, h->sys.n, x, &dx, true, st));
    TRY(stage(h, &h->d_ystage, h->sys.m, y, &dy, true, st));
    CK(launch_aprod1_f32_api(h, dx, dy, st));
    if (dy != y) {
        CK(cudaMemcpyAsync(y, dy, h->sys.m * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return GSR_OK;
}

extern "C" int gsr_aprod2_f32(void *hv, const double *y, double *x, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !x || !y)
        return GSR_ERR_ARG;
    if (h->cfg.precision != GSR_PREC_MIXED)
        return GSR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    double *dx, *dy;
    TRY(stage(h, &h->d_ystage, h->sys.m, y, &dy, true, st));
    TRY(stage(h, &h->d_xstage, h->sys.n, x, &dx, true, st));
    CK(launch_aprod2_f32_api(h, dy, dx, st));
    if (dx != x) {
        CK(cudaMemcpyAsync(x, dx, h->sys.n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return GSR_OK;
}

extern "C" int gsr_mixed_solve(void *hv, const double *b, int max_outer, int max_inner,
                               double inner_tol, double atol, double *x, gsr_mixed_result *out,
                               void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !b || !x || max_outer < 0 || max_inner < 1 || !(inner_tol >= 0.0) || !(atol >= 0.0))
        return GSR_ERR_ARG;
    if (h->cfg.precision != GSR_PREC_MIXED)
        return GSR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const SysView &A = h->sys;
    double *db;
    TRY(stage(h, &h->d_bstage, A.m, b, &db, true, st));
    CK(enqueue_precondition(h, h->d_p, st));
    CK(cudaMemsetAsync(h->d_xm, 0, A.n * sizeof(double), st));
    CK(cudaMemcpyAsync(h->d_r, db, A.m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    h->h_cgargs->max_inner = max_inner;
    h->h_cgargs->tol = inner_tol;
    CK(cudaMemcpyAsync(h->d_cgargs, h->h_cgargs, sizeof(CgArgs), cudaMemcpyHostToDevice, st));
    const double anorm = sqrt(h->n_nonempty);
    gsr_mixed_result res = {};
    res.anorm = anorm;
    for (int k = 0;; k++) {
        // FP64 normal residual c = A^T r and the stopping rule
        CK(cudaMemsetAsync(h->d_c, 0, A.n * sizeof(double), st));
        CK(launch_aprod2(h, h->d_r, h->d_c, kA2Accumulate, st));
        CK(launch_outer_norms(h, h->d_r, st));
        CK(cudaMemcpyAsync(h->h_onorm, h->d_onorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        res.arnorm = sqrt(h->h_onorm[0]);
        res.rnorm = sqrt(h->h_onorm[1]);
        if (!isfinite(res.arnorm) || !isfinite(res.rnorm))
            return GSR_ERR_NONFINITE;
        if (res.arnorm <= atol * anorm * res.rnorm) {
            res.converged = 1;
            break;
        }
        if (k >= max_outer)
            break;
        // inner CG on (diag(p) A32^T A32 diag(p)) z = p o c, then x += p o z
        CK(run_cg(h, st, max_inner));
        CK(cudaMemcpyAsync(h->h_cg, h->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, st));
        // r = b - A x in FP64
        CK(cudaMemcpyAsync(h->d_r, db, A.m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(launch_neg(h, h->d_xm, h->d_xneg, A.n, st));
        CK(launch_aprod1(h, h->d_xneg, h->d_r, 0, st));
        CK(cudaStreamSynchronize(st));
        if (h->h_cg->nonfinite)
            return GSR_ERR_NONFINITE;
        res.outer = k + 1;
        res.inner += h->h_cg->it;
    }
    CK(cudaMemcpyAsync(x, h->d_xm, A.n * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    TRY(take_kernel_status(h, st));
    if (out)
        *out = res;
    return GSR_OK;
}

extern "C" int gsr_product_forms(void *hv, int *aprod1_split_on, int *aprod2_split_on)
{
    const gsr_handle_t *h = (const gsr_handle_t *)hv;
    if (!h || !aprod1_split_on || !aprod2_split_on)
        return GSR_ERR_ARG;
    *aprod1_split_on = !aprod1_split(h) ? 0
                       : (h->a1_tma && (split_request(h->cfg) & GSR_SPLIT_APROD1_ASTRO)) ? 2 : 1;
    *aprod2_split_on = aprod2_split_active(h);
    return GSR_OK;
}

extern "C" int gsr_set_values(void *hv, int k, const double *values, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !values || k < 0 || k >= kNPar)
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *dv;
    TRY(stage(h, &h->d_ystage, h->sys.m, values, &dv, true, st));
    CK(launch_set_plane(h, k, dv, st));
    if (h->cfg.precision == GSR_PREC_MIXED)
        CK(launch_f32_plane(h, k, st));
    if (dv != values)
        CK(cudaStreamSynchronize(st));
    return GSR_OK;
}

// (diag(p) A^T A diag(p)) z = diag(p) g by FP64 CG, q = p o z, into h->d_xm
static int normal_solve_dev(gsr_handle_t *h, const double *dg, int max_iter, double tol,
                            gsr_cg_result *res, cudaStream_t st)
{
    const SysView &A = h->sys;
    CK(enqueue_precondition(h, h->d_p, st));
    CK(cudaMemcpyAsync(h->d_c, dg, A.n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(h->d_xm, 0, A.n * sizeof(double), st));
    h->h_cgargs->max_inner = max_iter;
    h->h_cgargs->tol = tol;
    CK(cudaMemcpyAsync(h->d_cgargs, h->h_cgargs, sizeof(CgArgs), cudaMemcpyHostToDevice, st));
    CK(run_cg64(h, st, max_iter));
    CK(cudaMemcpyAsync(h->h_cg, h->d_cg, sizeof(CgState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const CgState &g = *h->h_cg;
    if (res) {
        res->iterations = g.it;
        res->converged = (g.gamma <= g.stop2) ? 1 : 0;
        res->rel_resid = (g.gamma0 > 0.0) ? sqrt(g.gamma / g.gamma0) : 0.0;
    }
    if (g.nonfinite)
        return GSR_ERR_NONFINITE;
    return GSR_OK;
}

extern "C" int gsr_normal_solve(void *hv, const double *g, int max_iter, double tol, double *q,
                                gsr_cg_result *out, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !g || !q || max_iter < 1 || !(tol >= 0.0))
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double *dg;
    TRY(stage(h, &h->d_xstage, h->sys.n, g, &dg, true, st));
    TRY(normal_solve_dev(h, dg, max_iter, tol, out, st));
    CK(cudaMemcpyAsync(q, h->d_xm, h->sys.n * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    TRY(take_kernel_status(h, st));
    return GSR_OK;
}

extern "C" int gsr_lsq_backward(void *hv, const double *b, const double *x, const double *gx,
                                int max_iter, double tol, double *grad_b, double *grad_glob,
                                gsr_cg_result *out, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !b || !x || !gx || !grad_b || max_iter < 1 || !(tol >= 0.0))
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const SysView &A = h->sys;
    double *dgx, *dgb, *db, *dx;
    TRY(stage(h, &h->d_xstage, A.n, gx, &dgx, true, st));
    TRY(normal_solve_dev(h, dgx, max_iter, tol, out, st));  // q in d_xm
    // s = A q = dL/db
    TRY(stage(h, &h->d_ystage, A.m, grad_b, &dgb, false, st));
    CK(cudaMemsetAsync(dgb, 0, A.m * sizeof(double), st));
    CK(launch_aprod1(h, h->d_xm, dgb, 0, st));
    if (grad_glob) {
        // r = b - A x, then grad_glob = r q_G - s x_G
        TRY(stage(h, &h->d_bstage, A.m, b, &db, true, st));
        if (on_device(x)) {
            dx = (double *)x;
        } else {
            CK(cudaMemcpyAsync(h->d_xneg, x, A.n * sizeof(double), cudaMemcpyHostToDevice, st));
            dx = h->d_xneg;
        }
        CK(cudaMemcpyAsync(h->d_r, db, A.m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(launch_neg(h, dx, h->d_t, A.n, st));
        CK(launch_aprod1(h, h->d_t, h->d_r, 0, st));
        double *dgg = grad_glob;
        const bool gg_dev = on_device(grad_glob);
        if (!gg_dev)
            dgg = h->d_q64;  // m doubles of scratch
        CK(launch_grad_global(h, h->d_r, dgb, h->d_xm, dx, dgg, st));
        if (!gg_dev)
            CK(cudaMemcpyAsync(grad_glob, dgg, A.m * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (dgb != grad_b)
        CK(cudaMemcpyAsync(grad_b, dgb, A.m * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    TRY(take_kernel_status(h, st));
    return GSR_OK;
}

// buffers of the batched solve for k columns (leading dimension rounded up
// to 8 so that the column-tile loads are aligned) and its inner graph
static int ensure_batched(gsr_handle_t *h, int k)
{
    const SysView &A = h->sys;
    const int ldk = (k + 7) / 8 * 8;
    if (ldk > h->bk) {
        void *old[] = {h->d_bX32, h->d_bQ32, h->d_bC, h->d_bS_, h->d_bD, h->d_bZ, h->d_bT};
        for (void *p : old)
            if (p)
                cudaFree(p);
        h->d_bX32 = nullptr; h->d_bQ32 = nullptr; h->d_bC = nullptr; h->d_bS_ = nullptr;
        h->d_bD = nullptr; h->d_bZ = nullptr; h->d_bT = nullptr;
        TRY(dalloc(h, &h->d_bX32, A.n * ldk));
        TRY(dalloc(h, &h->d_bQ32, A.m * ldk));
        TRY(dalloc(h, &h->d_bC, A.n * ldk));
        TRY(dalloc(h, &h->d_bS_, A.n * ldk));
        TRY(dalloc(h, &h->d_bD, A.n * ldk));
        TRY(dalloc(h, &h->d_bZ, A.n * ldk));
        TRY(dalloc(h, &h->d_bT, A.n * ldk));
        h->bk = ldk;
    }
    if (!h->d_bS) {
        TRY(dalloc(h, &h->d_bS, A.nseg * kNAtt * 8));
        TRY(dalloc(h, &h->d_bipart, A.I * 4 * 8));
        TRY(dalloc(h, &h->d_bpartial, (int64_t)8 * kMaxPartials));
        TRY(dalloc(h, &h->d_bcounter, 1));
        TRY(dalloc(h, &h->d_bs, 1));
        TRY(dalloc(h, &h->d_bargs, 1));
        TRY(dalloc(h, &h->d_bnorms, 2 * kMaxBatch));
        CK(cudaMemset(h->d_bcounter, 0, sizeof(unsigned)));
        CK(cudaMallocHost((void **)&h->h_bs, sizeof(BatchState)));
        CK(cudaMallocHost((void **)&h->h_bargs, sizeof(BatchArgs)));
        CK(cudaMallocHost((void **)&h->h_bnorms, 2 * kMaxBatch * sizeof(double)));
        h->grid_b1 = batched_grid_rows(h);
        h->grid_b2 = batched_grid_stars(h);
        if (h->grid_b1 <= 0 || h->grid_b2 <= 0)
            return cuda_fail(cudaGetLastError(), "batched occupancy");
    }
    if (!h->b_exec || h->b_graph_k != h->bk || h->b_graph_kt != h->b_kt ||
        h->b_graph_lanes != h->b_lanes) {
        cudaError_t e = build_batched_graph(h, h->bk);
        if (e != cudaSuccess)
            return cuda_fail(e, "build_batched_graph");
    }
    return GSR_OK;
}

static int cm_buffers(gsr_handle_t *h, int k)
{
    const SysView &A = h->sys;
    if (h->d_bXcm && h->bkcm == k)
        return GSR_OK;
    void *old[] = {h->d_bXcm, h->d_bCcm};
    for (void *p : old)
        if (p)
            cudaFree(p);
    h->d_bXcm = h->d_bCcm = nullptr;
    TRY(dalloc(h, &h->d_bXcm, A.n * k));
    TRY(dalloc(h, &h->d_bCcm, A.n * k));
    h->bkcm = k;
    return GSR_OK;
}

extern "C" int gsr_set_aprod2_fused(void *hv, int fused)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || (fused != 0 && fused != 1))
        return GSR_ERR_ARG;
    if (h->ipath != kIpSorted)
        return GSR_ERR_UNSUPPORTED;
    if (h->a2_fused == fused)
        return GSR_OK;
    h->a2_fused = fused;
    // the captured graphs hold the old launches: capture them again
    if (h->solve_exec) {
        cudaGraphExecDestroy(h->solve_exec);
        h->solve_exec = nullptr;
    }
    if (h->cg64_exec) {
        cudaGraphExecDestroy(h->cg64_exec);
        h->cg64_exec = nullptr;
    }
    const bool mixed = h->cg_exec != nullptr;
    if (h->cg_exec) {
        cudaGraphExecDestroy(h->cg_exec);
        h->cg_exec = nullptr;
    }
    cudaError_t e = build_solve_graph(h);
    if (e == cudaSuccess)
        e = build_cg64_graph(h);
    if (e == cudaSuccess && mixed)
        e = build_cg_graph(h);
    if (e != cudaSuccess)
        return cuda_fail(e, "gsr_set_aprod2_fused");
    return GSR_OK;
}

// the captured graphs hold the old launches: capture them again
static int recapture_graphs(gsr_handle_t *h, const char *what)
{
    if (h->solve_exec) {
        cudaGraphExecDestroy(h->solve_exec);
        h->solve_exec = nullptr;
    }
    if (h->cg64_exec) {
        cudaGraphExecDestroy(h->cg64_exec);
        h->cg64_exec = nullptr;
    }
    const bool mixed = h->cg_exec != nullptr;
    if (h->cg_exec) {
        cudaGraphExecDestroy(h->cg_exec);
        h->cg_exec = nullptr;
    }
    cudaError_t e = build_solve_graph(h);
    if (e == cudaSuccess)
        e = build_cg64_graph(h);
    if (e == cudaSuccess && mixed)
        e = build_cg_graph(h);
    if (e != cudaSuccess)
        return cuda_fail(e, what);
    return GSR_OK;
}

extern "C" int gsr_set_aprod1_staging(void *hv, int staged)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || (staged != 0 && staged != 1))
        return GSR_ERR_ARG;
    if (staged && !h->a1_tma_avail)
        return GSR_ERR_UNSUPPORTED;
    if (h->a1_tma == staged)
        return GSR_OK;
    const int old_tma = h->a1_tma, old_grid = h->grid_rows;
    h->a1_tma = staged;
    const int g = aprod1_grid(h);
    if (g <= 0 || g > kMaxPartials) {
        h->a1_tma = old_tma;
        h->grid_rows = old_grid;
        return cuda_fail(cudaGetLastError(), "gsr_set_aprod1_staging");
    }
    h->grid_rows = g;
    return recapture_graphs(h, "gsr_set_aprod1_staging");
}

extern "C" int gsr_aprod1_staging(void *hv, int *staged)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !staged)
        return GSR_ERR_ARG;
    *staged = h->a1_tma;
    return GSR_OK;
}

extern "C" int gsr_inject_missing_copy(void *hv, int64_t tile)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || tile < -1)
        return GSR_ERR_ARG;
    h->drop_tile = tile;
    return recapture_graphs(h, "gsr_inject_missing_copy");
}

extern "C" int gsr_set_batch_tiling(void *hv, int kt, int lanes)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || (kt != 1 && kt != 2 && kt != 4 && kt != 8) || (lanes != 8 && lanes != 16 && lanes != 32))
        return GSR_ERR_ARG;
    h->b_kt = kt;
    h->b_lanes = lanes;
    return GSR_OK;
}

extern "C" int gsr_batched_products(void *hv, int k, const double *X, const double *Y, double *Q,
                                    double *T, void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !X || !Y || !Q || !T || k < 1 || k > kMaxBatch)
        return GSR_ERR_ARG;
    if (h->cfg.precision != GSR_PREC_MIXED)
        return GSR_ERR_UNSUPPORTED;
    if (!on_device(X) || !on_device(Y) || !on_device(Q) || !on_device(T))
        return GSR_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const SysView &A = h->sys;
    TRY(ensure_batched(h, k));
    CK(cudaMemsetAsync(h->d_bX32, 0, A.n * h->bk * sizeof(float), st));
    CK(cudaMemsetAsync(h->d_bQ32, 0, A.m * h->bk * sizeof(float), st));
    CK(launch_b_layout(h, 1, X, h->d_bX32, 1, A.n, k, st));
    // Y goes into the binary32 m-block; Q32 is produced into d_bX32's partner
    float *Y32 = h->d_bQ32;
    CK(launch_b_layout(h, 1, Y, Y32, 1, A.m, k, st));
    // T = A32^T Y needs Y32 intact while Q = A32 X is formed: use d_bC as the
    // row-major FP64 T, and a second binary32 m-block for Q
    float *Q32 = nullptr;
    if (cudaMalloc(&Q32, A.m * h->bk * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return GSR_ERR_OOM;
    }
    cudaError_t e = cudaMemsetAsync(h->d_bC, 0, A.n * h->bk * sizeof(double), st);
    if (e == cudaSuccess)
        e = launch_b_products(h, h->bk, h->d_bX32, Q32, Y32, h->d_bC, st);
    if (e == cudaSuccess)
        e = launch_b_layout(h, 0, (const double *)Q32, Q, 2, A.m, k, st);
    if (e == cudaSuccess)
        e = launch_b_layout(h, 0, h->d_bC, T, 0, A.n, k, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaFree(Q32);
    if (e != cudaSuccess)
        return cuda_fail(e, "gsr_batched_products");
    return GSR_OK;
}

extern "C" int gsr_batched_solve(void *hv, int k, const double *B, int max_outer, int max_inner,
                                 double inner_tol, double atol, double *X, gsr_mixed_result *out,
                                 void *stream)
{
    gsr_handle_t *h = (gsr_handle_t *)hv;
    if (!h || !B || !X || k < 1 || k > kMaxBatch || max_outer < 0 || max_inner < 1 ||
        !(inner_tol >= 0.0) || !(atol >= 0.0))
        return GSR_ERR_ARG;
    if (h->cfg.precision != GSR_PREC_MIXED)
        return GSR_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const SysView &A = h->sys;
    TRY(ensure_batched(h, k));
    TRY(cm_buffers(h, k));
    // right-hand sides: the caller's device block in place, or a staged copy
    const double *dB = B;
    if (!on_device(B)) {
        if (h->bkB < k) {
            if (h->d_bB)
                cudaFree(h->d_bB);
            h->d_bB = nullptr;
            h->bkB = 0;
            TRY(dalloc(h, &h->d_bB, A.m * k));
            h->bkB = k;
        }
        CK(cudaMemcpyAsync(h->d_bB, B, A.m * k * sizeof(double), cudaMemcpyHostToDevice, st));
        dB = h->d_bB;
    }
    CK(enqueue_precondition(h, h->d_p, st));
    CK(cudaMemsetAsync(h->d_bXcm, 0, A.n * k * sizeof(double), st));
    h->h_bargs->max_inner = max_inner;
    h->h_bargs->tol = inner_tol;
    CK(cudaMemcpyAsync(h->d_bargs, h->h_bargs, sizeof(BatchArgs), cudaMemcpyHostToDevice, st));
    const double anorm = sqrt(h->n_nonempty);
    std::vector<gsr_mixed_result> res((size_t)k);
    for (int c = 0; c < k; c++)
        res[c].anorm = anorm;
    for (int it = 0;; it++) {
        // FP64 residual r_c = b_c - A x_c and normal residual c_c = A^T r_c,
        // one column at a time through one m-vector
        CK(cudaMemsetAsync(h->d_bCcm, 0, A.n * k * sizeof(double), st));
        for (int c = 0; c < k; c++) {
            const double *bc = dB + (int64_t)c * A.m;
            const double *r = bc;  // x = 0 on the first pass
            if (it > 0) {
                CK(cudaMemcpyAsync(h->d_r, bc, A.m * sizeof(double), cudaMemcpyDeviceToDevice, st));
                CK(launch_neg(h, h->d_bXcm + (int64_t)c * A.n, h->d_xneg, A.n, st));
                CK(launch_aprod1(h, h->d_xneg, h->d_r, 0, st));
                r = h->d_r;
            }
            CK(launch_aprod2(h, r, h->d_bCcm + (int64_t)c * A.n, kA2Accumulate, st));
            CK(launch_norms2(h, h->d_bCcm + (int64_t)c * A.n, r, h->d_bnorms + 2 * c, st));
        }
        CK(cudaMemcpyAsync(h->h_bnorms, h->d_bnorms, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (it > 0 && h->h_bs->nonfinite)
            return GSR_ERR_NONFINITE;
        int all = 1;
        for (int c = 0; c < k; c++) {
            res[c].arnorm = sqrt(h->h_bnorms[2 * c]);
            res[c].rnorm = sqrt(h->h_bnorms[2 * c + 1]);
            if (!isfinite(res[c].arnorm) || !isfinite(res[c].rnorm))
                return GSR_ERR_NONFINITE;
            res[c].converged = res[c].arnorm <= atol * anorm * res[c].rnorm;
            all &= res[c].converged;
        }
        if (all || it >= max_outer)
            break;
        // inner solve of all columns (converged ones have a tiny right-hand side)
        CK(cudaMemsetAsync(h->d_bC, 0, A.n * h->bk * sizeof(double), st));
        CK(launch_b_layout(h, 1, h->d_bCcm, h->d_bC, 0, A.n, k, st));
        CK(run_batched_inner(h, h->bk, max_inner, st));
        CK(launch_b_update_x(h, h->d_bXcm, k, st));
        CK(cudaMemcpyAsync(h->h_bs, h->d_bs, sizeof(BatchState), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int c = 0; c < k; c++) {
            res[c].outer = it + 1;
            res[c].inner += h->h_bs->it[c];
        }
    }
    CK(cudaMemcpyAsync(X, h->d_bXcm, A.n * k * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    TRY(take_kernel_status(h, st));
    if (out)
        for (int c = 0; c < k; c++)
            out[c] = res[c];
    return GSR_OK;
}
