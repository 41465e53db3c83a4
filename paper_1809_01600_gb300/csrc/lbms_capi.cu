// C ABI of the solver (declared in include/lbms.h): validation, host
// properties, fluid-cell indexing, batching of cases into one index space,
// device state, tile autotuning, CUDA-graph stepping, residual loops and
// the FP64 post-processing of Eq. 43.  A single-case solver is a batch of 1.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbms.h"
#include "lbms_internal.h"
#include "lbms_kernels.cuh"
#include "lbms_lattice.cuh"
#include "lbms_props.cuh"

using namespace lbms;

namespace {

struct CaseHost {
    int nx = 0, ny = 0, nz = 0, periodic_x = 0;
    int64_t N = 0;
    double length_x = 0.0;
    std::vector<int64_t> fluid_cell;  // dense index of each fluid cell, x-fastest order
    int base = 0, nf = 0;             // range [base, base + nf) of the kernels' index space
    int wpr = 0, tab = 0;             // row-bitmask table: entries per row, first entry of the case
    int row_first = 0, nrows = 0;     // rows (y, z) in the concatenated row lists
    double dx = 0.0, dt = 0.0;
    double x_in[3] = {0, 0, 0};
    double current = 0.0;
    double q[3] = {0, 0, 0};          // outlet flux per node per step (lattice units)
    bool has_bc = false;
};

}  // namespace

struct lbms_ctx {
    int dim = 2, Q = 9;
    std::vector<CaseHost> cases;
    GasProps gas{};                   // D_eff, C_t, T, p, stoichiometry (dx, dt are per case)
    lbms_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    Launch L;
    std::vector<std::pair<void*, size_t>> allocs;
    size_t device_bytes = 0;
    double* host_out = nullptr;       // pinned, cases * kCaseOutSlots doubles
    std::vector<unsigned char> case_bc;  // packed CaseBC images of all cases
    bool initialized = false;         // every case has boundary data
    bool tuned = false;
    int64_t steps = 0;
    uint64_t h2d = 0, d2h = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::string err;
};

namespace {

constexpr int kGraphSteps = 32;  // even: a replay returns to the same parity

thread_local std::string t_create_error;  // message of the last failed lbms_create on this thread

lbms_status fail(lbms_ctx* c, lbms_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

lbms_status cuda_fail(lbms_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? LBMS_ENOMEM : LBMS_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(call, what)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

void* dev_alloc(lbms_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->opt.alloc) {
        p = c->opt.alloc(bytes, c->stream, c->opt.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) {
        c->allocs.emplace_back(p, bytes);
        c->device_bytes += bytes;
    }
    return p;
}

// Releases one allocation of dev_alloc before the handle's end.
void dev_free(lbms_ctx* c, void* p) {
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (c->allocs[k].first != p) continue;
        cudaStreamSynchronize(c->stream);
        if (c->opt.free)
            c->opt.free(p, c->allocs[k].second, c->stream, c->opt.alloc_user);
        else
            cudaFree(p);
        c->device_bytes -= c->allocs[k].second;
        c->allocs.erase(c->allocs.begin() + (std::ptrdiff_t)k);
        return;
    }
}

void drop_graphs(lbms_ctx* c) {
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
}

void release(lbms_ctx* c) {
    drop_graphs(c);
    if (!c->allocs.empty()) cudaStreamSynchronize(c->stream);
    for (auto& a : c->allocs) {
        if (c->opt.free)
            c->opt.free(a.first, a.second, c->stream, c->opt.alloc_user);
        else
            cudaFree(a.first);
    }
    c->allocs.clear();
    if (c->host_out) cudaFreeHost(c->host_out);
    c->host_out = nullptr;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->cap_stream = nullptr;
}

// Eqs. 40-42 and C_t; the lattice diffusivities follow from the time-step
// policy (or the explicit dt of the options and the first case's spacing).
lbms_status compute_props(lbms_ctx* c, const lbms_species* sp, const lbms_diffusivities* df, double T, double p) {
    GasProps& g = c->gas;
    g.T = T;
    g.p = p;
    g.electrons = sp->electrons;
    for (int s = 0; s < 3; ++s) g.stoich[s] = sp->stoich[s];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i == j) {
                g.D_bin[i][j] = 0.0;
                continue;
            }
            if (df && df->D_binary_m2s)
                g.D_bin[i][j] = df->D_binary_m2s[i * 3 + j];
            else
                g.D_bin[i][j] = 1.0e-4 * fuller_cm2s(T, p, sp->molar_mass[i], sp->molar_mass[j],
                                                     sp->fuller_volume[i], sp->fuller_volume[j]);
            if (!(g.D_bin[i][j] > 0.0) || !std::isfinite(g.D_bin[i][j]))
                return fail(c, LBMS_EINVAL, "binary diffusivity D[%d][%d] must be finite and > 0", i, j);
        }
    const double dp = df ? df->pore_diameter_m : 0.0;
    const double phi = df ? df->eps_over_tau : 1.0;
    if (!(phi > 0.0) || !std::isfinite(phi)) return fail(c, LBMS_EINVAL, "eps_over_tau must be finite and > 0");
    for (int i = 0; i < 3; ++i)
        g.D_kn[i] = dp > 0.0 ? knudsen_m2s(T, sp->molar_mass[i], dp) : std::numeric_limits<double>::infinity();
    double dmin = std::numeric_limits<double>::infinity();
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (i == j) {
                g.D_eff[i][j] = 0.0;
                continue;
            }
            const double a = 1.0 / (1.0 / g.D_bin[i][j] + 1.0 / g.D_kn[i]);
            const double b = 1.0 / (1.0 / g.D_bin[i][j] + 1.0 / g.D_kn[j]);
            g.D_eff[i][j] = 0.5 * phi * (a + b);
            dmin = std::min(dmin, g.D_eff[i][j]);
        }
    g.C_t = p / (kR * T);
    for (auto& cs : c->cases) {
        cs.dx = cs.periodic_x ? cs.length_x / cs.nx : cs.length_x / (cs.nx - 1);
        cs.dt = c->opt.dt_s > 0.0 ? c->opt.dt_s : cs.dx * cs.dx / (6.0 * dmin);
    }
    const CaseHost& c0 = c->cases[0];
    for (const auto& cs : c->cases)
        if (std::fabs(cs.dt / (cs.dx * cs.dx) - c0.dt / (c0.dx * c0.dx)) > 1e-12 * c0.dt / (c0.dx * c0.dx))
            return fail(c, LBMS_EINVAL, "an explicit dt_s needs the same grid spacing in every case");
    g.dx = c0.dx;
    g.dt = c0.dt;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) g.D_lat[i][j] = g.D_eff[i][j] * c0.dt / (c0.dx * c0.dx);
    return LBMS_OK;
}

lbms_status validate_bc(lbms_ctx* c, const double* x, double I) {
    if (!x) return fail(c, LBMS_EINVAL, "x_inlet is NULL");
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
        if (!(x[i] >= 0.0) || !std::isfinite(x[i])) return fail(c, LBMS_EINVAL, "x_inlet[%d] must be finite and >= 0", i);
        s += x[i];
    }
    if (std::fabs(s - 1.0) > 1e-9) return fail(c, LBMS_EINVAL, "x_inlet must sum to 1 (got %.12g)", s);
    if (!(I >= 0.0) || !std::isfinite(I)) return fail(c, LBMS_EINVAL, "current density must be finite and >= 0");
    return LBMS_OK;
}

// Uploads the device CaseBC entry of case k (inlet values, outlet flux, range).
lbms_status upload_case_bc(lbms_ctx* c, int k) {
    const CaseHost& cs = c->cases[k];
    CaseHostBC h;
    for (int s = 0; s < 3; ++s) {
        h.xin[s] = cs.x_in[s];
        h.q[s] = cs.q[s];
    }
    h.base = cs.base;
    h.nf = cs.nf;
    h.nx = cs.nx;
    h.ny = cs.ny;
    h.nz = cs.nz;
    h.wpr = cs.wpr;
    h.tab = cs.tab;
    const size_t sz = case_bc_size(c->L.precision);
    pack_case_bc(c->L.precision, h, c->case_bc.data() + k * sz);
    CK(cudaMemcpyAsync(static_cast<unsigned char*>(c->L.b.cases) + k * sz, c->case_bc.data() + k * sz, sz,
                       cudaMemcpyHostToDevice, c->stream),
       "upload boundary data");
    c->h2d += sz;
    return LBMS_OK;
}

// Mole fractions in the device format: double, or a double-float pair whose
// hi word is at [s][i] and lo word at [3 + s][i] (idx = s * S + i).
void put_x(int precision, unsigned char* buf, int64_t S, int64_t idx, double v) {
    if (precision == LBMS_FP64) {
        reinterpret_cast<double*>(buf)[idx] = v;
    } else {
        const float hi = (float)v;
        reinterpret_cast<float*>(buf)[idx] = hi;
        reinterpret_cast<float*>(buf)[idx + 3 * S] = (float)(v - (double)hi);
    }
}

double get_x(int precision, const unsigned char* buf, int64_t S, int64_t idx) {
    if (precision == LBMS_FP64) return reinterpret_cast<const double*>(buf)[idx];
    return (double)reinterpret_cast<const float*>(buf)[idx] + (double)reinterpret_cast<const float*>(buf)[idx + 3 * S];
}

// Rows (species, and hi/lo words) of the X buffer as a pitched 2-D region.
int x_rows(int precision) { return precision == LBMS_FP64 ? 3 : 6; }
size_t x_word(int precision) { return precision == LBMS_FP64 ? sizeof(double) : sizeof(float); }

// Chooses the step kernel's tile shape by timing each variant on the real
// state: the variants read lattice cur and write lattice cur ^ 1 without
// swapping, so the state is unchanged; the X copy of cur ^ 1 is restored.
lbms_status autotune(lbms_ctx* c) {
    Launch& L = c->L;
    if (c->opt.step_variant > 0) {
        const int v = c->opt.step_variant - 1;
        if (kVariantNb[v] == kNbOffset16 && !L.b.nbr16)
            return fail(c, LBMS_EINVAL, "step variant %d needs the 16-bit neighbour table, which was not built", v);
        if (kVariantNb[v] == kNbRowMask && !L.b.rowtab)
            return fail(c, LBMS_EINVAL,
                        "step variant %d needs the row-bitmask tables (no box periodic in x, nx <= %d, ny <= %d, "
                        "nz <= %d)",
                        v, kRowMaskMaxNx, kRowMaskMaxNy, kRowMaskMaxNz);
        L.variant = v;
        c->tuned = true;
        return LBMS_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "autotune event");
    CK(cudaEventCreate(&e1), "autotune event");
    float best = std::numeric_limits<float>::infinity();
    int pick = L.outlet_extrap ? 6 : 0;
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < kStepVariants && e == cudaSuccess; ++v) {
        if (kVariantNb[v] == kNbOffset16 && !L.b.nbr16) continue;
        if (kVariantNb[v] == kNbRowMask && !L.b.rowtab) continue;
        if (L.outlet_extrap && !kVariantPerCell[v]) continue;   // the per-cell kernel alone has it
        e = launch_step_variant(L, v, c->stream);  // warm-up
        if (e != cudaSuccess) break;
        e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_step_variant(L, v, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
            best = ms;
            pick = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
    L.variant = pick;
    const size_t xbytes = (size_t)3 * L.S * x_size(L.precision);
    CK(cudaMemcpyAsync(L.b.X[L.cur ^ 1], L.b.X[L.cur], xbytes, cudaMemcpyDeviceToDevice, c->stream), "autotune restore");
    CK(cudaStreamSynchronize(c->stream), "autotune");
    c->tuned = true;
    return LBMS_OK;
}

// Copies a dense host field of case k (3 * N doubles) into X[cur] and
// restarts that case from the equilibrium f = w X (h = 0).
lbms_status upload_field(lbms_ctx* c, int k, const double* X) {
    CaseHost& cs = c->cases[k];
    const int prec = c->L.precision;
    const int64_t S = c->L.S;
    const int rows = x_rows(prec);
    const size_t word = x_word(prec);
    // a compact [rows][nf] image of the case's slice, copied as a pitched region
    std::vector<unsigned char> buf((size_t)rows * cs.nf * word, 0);
    for (int s = 0; s < 3; ++s)
        for (int i = 0; i < cs.nf; ++i) put_x(prec, buf.data(), cs.nf, (int64_t)s * cs.nf + i, X[(size_t)s * cs.N + cs.fluid_cell[i]]);
    unsigned char* dst = static_cast<unsigned char*>(c->L.b.X[c->L.cur]) + (size_t)cs.base * word;
    CK(cudaMemcpy2DAsync(dst, S * word, buf.data(), cs.nf * word, cs.nf * word, rows, cudaMemcpyHostToDevice, c->stream),
       "upload mole fractions");
    c->h2d += buf.size();
    CK(launch_init(c->L, cs.base, cs.nf, c->stream), "init kernel");
    CK(cudaStreamSynchronize(c->stream), "init");
    return LBMS_OK;
}

// Initial state of Section 4.1: with the fluxes held at their outlet values
// N_i = -nu_i I / (n F) (Eq. 39) across the anode, Eq. 19 (Gamma = I),
//   dX_i/dx = sum_{j != i} (X_i N_j - X_j N_i) / (C_t D_ij,eff),
// is integrated from X_in at x = 0 to every node x_j = j dx (classical
// fourth-order Runge-Kutta, 16 substeps per node spacing).  prof[s * nx + j].
// False if a mole fraction goes negative (the current depletes a reactant).
bool profile_1d(const GasProps& g, const CaseHost& cs, double current, std::vector<double>& prof) {
    const double I = current * 1.0e4;
    double N[3];
    for (int s = 0; s < 3; ++s) N[s] = -g.stoich[s] * I / (g.electrons * kF);
    auto rhs = [&](const double* X, double* dX) {
        for (int i = 0; i < 3; ++i) {
            double v = 0.0;
            for (int j = 0; j < 3; ++j)
                if (j != i) v += (X[i] * N[j] - X[j] * N[i]) / (g.C_t * g.D_eff[i][j]);
            dX[i] = v;
        }
    };
    constexpr int kSub = 16;
    const double h = cs.dx / kSub;
    prof.assign(3 * (size_t)cs.nx, 0.0);
    double X[3] = {cs.x_in[0], cs.x_in[1], cs.x_in[2]};
    for (int j = 0; j < cs.nx; ++j) {
        for (int s = 0; s < 3; ++s) {
            if (!(X[s] >= 0.0)) return false;
            prof[(size_t)s * cs.nx + j] = X[s];
        }
        for (int m = 0; m < kSub && j + 1 < cs.nx; ++m) {
            double k1[3], k2[3], k3[3], k4[3], t[3];
            rhs(X, k1);
            for (int s = 0; s < 3; ++s) t[s] = X[s] + 0.5 * h * k1[s];
            rhs(t, k2);
            for (int s = 0; s < 3; ++s) t[s] = X[s] + 0.5 * h * k2[s];
            rhs(t, k3);
            for (int s = 0; s < 3; ++s) t[s] = X[s] + h * k3[s];
            rhs(t, k4);
            for (int s = 0; s < 3; ++s) X[s] += h / 6.0 * (k1[s] + 2.0 * k2[s] + 2.0 * k3[s] + k4[s]);
        }
    }
    return true;
}

lbms_status set_case_bc(lbms_ctx* c, int k, const double* x_inlet, double current) {
    lbms_status st = validate_bc(c, x_inlet, current);
    if (st != LBMS_OK) return st;
    CaseHost& cs = c->cases[k];
    for (int s = 0; s < 3; ++s) cs.x_in[s] = x_inlet[s];
    cs.current = current;
    if (cs.periodic_x) {
        for (int s = 0; s < 3; ++s) cs.q[s] = 0.0;
    } else {
        GasProps g = c->gas;
        g.dx = cs.dx;
        g.dt = cs.dt;
        outlet_flux_lattice(g, current, cs.q);
    }
    st = upload_case_bc(c, k);
    if (st != LBMS_OK) return st;
    if (!cs.has_bc) {
        std::vector<double> X(3 * (size_t)cs.N, 0.0);
        if (c->opt.init_mode == LBMS_INIT_PROFILE_1D && !cs.periodic_x) {
            std::vector<double> prof;
            if (!profile_1d(c->gas, cs, current, prof))
                return fail(c, LBMS_EDEPLETED, "the 1-D initial profile of case %d drives a mole fraction below zero", k);
            const int64_t plane = (int64_t)cs.ny * cs.nz;
            for (int s = 0; s < 3; ++s)
                for (int64_t r = 0; r < plane; ++r)
                    std::copy(prof.begin() + (size_t)s * cs.nx, prof.begin() + (size_t)(s + 1) * cs.nx,
                              X.begin() + s * cs.N + r * cs.nx);
        } else {
            for (int s = 0; s < 3; ++s) std::fill(X.begin() + s * cs.N, X.begin() + (s + 1) * cs.N, cs.x_in[s]);
        }
        st = upload_field(c, k, X.data());
        if (st != LBMS_OK) return st;
        cs.has_bc = true;
    }
    if (!c->initialized) {
        bool all = true;
        for (const auto& q : c->cases) all = all && q.has_bc;
        if (all) {
            c->initialized = true;
            c->steps = 0;
            if (!c->tuned) return autotune(c);
        }
    }
    return LBMS_OK;
}

lbms_status launch_steps(lbms_ctx* c, int64_t n) {
    while (n > 0) {
        if (n >= kGraphSteps) {
            const int par = c->L.cur;
            if (!c->graph[par]) {
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                Launch L = c->L;
                cudaError_t e = cudaSuccess;
                for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) {
                    e = launch_step(L, c->cap_stream);
                    L.cur ^= 1;
                }
                cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
                if (e != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return cuda_fail(c, e, "capture step launches");
                }
                if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
                e = cudaGraphInstantiate(&c->graph[par], g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    c->graph[par] = nullptr;
                    return cuda_fail(c, e, "instantiate step graph");
                }
            }
            CK(cudaGraphLaunch(c->graph[par], c->stream), "graph launch");
            n -= kGraphSteps;
            c->steps += kGraphSteps;
        } else {
            CK(launch_step(c->L, c->stream), "step kernel");
            c->L.cur ^= 1;
            --n;
            ++c->steps;
        }
    }
    return LBMS_OK;
}

// Reads n doubles of the per-case output buffer starting at offset.
lbms_status read_case_out(lbms_ctx* c, size_t offset, size_t n) {
    CK(cudaMemcpyAsync(c->host_out + offset, c->L.b.case_out + offset, n * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream),
       "reduction readback");
    CK(cudaStreamSynchronize(c->stream), "reduction");
    c->d2h += n * sizeof(double);
    return LBMS_OK;
}

// Per-case residuals (refreshing the snapshots); LBMS_EUNSTABLE on NaN/Inf.
lbms_status case_residuals(lbms_ctx* c, int K, double* r) {
    const int n = c->L.n_cases;
    CK(launch_case_residuals(c->L, 1, c->stream), "residual kernels");
    lbms_status st = read_case_out(c, 0, (size_t)n * 10);
    if (st != LBMS_OK) return st;
    bool bad = false;
    for (int k = 0; k < n; ++k) {
        const double* o = c->host_out + (size_t)k * 10;
        if (o[9] > 0.0) {
            r[k] = std::numeric_limits<double>::infinity();
            bad = true;
            continue;
        }
        double res = 0.0;
        for (int s = 0; s < 3; ++s)
            if (o[3 + s] > 0.0) res = std::max(res, std::sqrt(o[s]) / (K * std::sqrt(o[3 + s])));
        r[k] = res;
    }
    if (bad) return fail(c, LBMS_EUNSTABLE, "non-finite mole fractions after %lld steps", (long long)c->steps);
    return LBMS_OK;
}

lbms_status case_boundary(lbms_ctx* c) {
    CK(launch_case_boundary(c->L, c->stream), "boundary kernel");
    return read_case_out(c, (size_t)c->L.n_cases * 10, (size_t)c->L.n_cases * 6);
}

lbms_status overpotential_of(lbms_ctx* c, int k, double* eta, double* xo_out) {
    const CaseHost& cs = c->cases[k];
    const double* o = c->host_out + (size_t)c->L.n_cases * 10 + (size_t)k * 6;
    double xo[3];
    for (int s = 0; s < 3; ++s) xo[s] = o[3 + s] / cs.nrows;
    if (xo_out)
        for (int s = 0; s < 3; ++s) xo_out[s] = xo[s];
    const double a = cs.x_in[0] * xo[1];
    const double b = xo[0] * cs.x_in[1];
    if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b)) {
        if (eta) *eta = std::numeric_limits<double>::quiet_NaN();
        return fail(c, LBMS_EDEPLETED, "case %d: Eq. 43 undefined: X_in = (%g, %g), X_out = (%g, %g)", k, cs.x_in[0],
                    cs.x_in[1], xo[0], xo[1]);
    }
    if (eta) *eta = kR * c->gas.T / (c->gas.electrons * kF) * std::log(a / b);
    return LBMS_OK;
}

bool bad_case(const lbms_ctx* c, int k) { return !c || k < 0 || k >= (int)c->cases.size(); }

// Aitken extrapolation of the slowest decay mode, per case (see the
// extrapolate_every option).  norm_prev / rho_prev hold each case's last
// W-step change and ratio (negative: none yet).
struct Extrapolator {
    std::vector<double> norm_prev, rho_prev, coef;
    int64_t since = 0;
    int rre_n = 0;                     // snapshots taken in the current reduced-rank cycle
    std::vector<double> rre_coef;      // [cases][order]
    std::vector<int> polish;           // per case: 0 not yet at tol, 1 final extrapolation pending, 2 done
    std::vector<int> polish_n;         // final extrapolations taken per case
};

// The final extrapolation of a case repeats while its jump moved X by more
// than kPolishRel of |X| (it removes most, not all, of the slowest mode), at
// most kPolishMax times.
constexpr double kPolishRel = 1e-5;
constexpr int kPolishMax = 3;

lbms_status extrap_begin(lbms_ctx* c, Extrapolator& ex) {
    const int n = c->L.n_cases;
    if (!c->L.b.extrap) {
        c->L.b.extrap = static_cast<double*>(dev_alloc(c, (size_t)3 * c->L.S * sizeof(double)));
        if (!c->L.b.extrap) return fail(c, LBMS_ENOMEM, "extrapolation snapshot");
        CK(cudaMemsetAsync(c->L.b.extrap, 0, (size_t)3 * c->L.S * sizeof(double), c->stream), "extrapolation init");
    }
    ex.norm_prev.assign(n, -1.0);
    ex.rho_prev.assign(n, -1.0);
    ex.coef.assign(n, 0.0);
    ex.polish.assign(n, 0);
    ex.polish_n.assign(n, 0);
    ex.since = 0;
    // E = X (coefficient 0 leaves X alone)
    CK(cudaMemcpyAsync(c->L.b.coef, ex.coef.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "coef");
    CK(launch_extrapolate(c->L, c->stream), "extrapolation kernel");
    return LBMS_OK;
}

lbms_status extrap_check(lbms_ctx* c, Extrapolator& ex) {
    const int n = c->L.n_cases;
    CK(launch_case_extrap_norms(c->L, c->stream), "extrapolation norms");
    lbms_status st = read_case_out(c, 0, (size_t)n * 10);
    if (st != LBMS_OK) return st;
    for (int k = 0; k < n; ++k) {
        const double* o = c->host_out + (size_t)k * 10;
        const double nrm = std::sqrt(o[0] + o[1] + o[2]);
        double cf = 0.0;
        if (ex.polish[k] == 1 && ex.norm_prev[k] > 0.0 && std::isfinite(nrm)) {
            // the final extrapolation of a case that met tol: by now the slowest
            // mode dominates both W-step changes, so one ratio suffices
            const double rho = nrm / ex.norm_prev[k];
            if (rho > 0.05 && rho < 0.98) cf = rho / (1.0 - rho);
            const double xn = std::sqrt(o[3] + o[4] + o[5]);
            const bool again = cf > 0.0 && xn > 0.0 && cf * nrm > kPolishRel * xn && ++ex.polish_n[k] < kPolishMax;
            ex.polish[k] = again ? 1 : 2;
            ex.norm_prev[k] = -1.0;
            ex.rho_prev[k] = -1.0;
        } else if (ex.norm_prev[k] > 0.0 && std::isfinite(nrm)) {
            const double rho = nrm / ex.norm_prev[k];
            if (ex.rho_prev[k] > 0.0 && std::fabs(rho - ex.rho_prev[k]) <= 0.02 * rho && rho > 0.05 && rho < 0.98) {
                cf = rho / (1.0 - rho);
                ex.norm_prev[k] = -1.0;   // the jump breaks the geometric sequence
                ex.rho_prev[k] = -1.0;
            } else {
                ex.rho_prev[k] = rho;
                ex.norm_prev[k] = nrm;
            }
        } else {
            ex.norm_prev[k] = nrm;
        }
        ex.coef[k] = cf;
    }
    CK(cudaMemcpyAsync(c->L.b.coef, ex.coef.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "coef");
    c->h2d += n * sizeof(double);
    CK(launch_extrapolate(c->L, c->stream), "extrapolation kernel");
    ex.since = 0;
    return LBMS_OK;
}

// Reduced-rank extrapolation (extrapolate_modes = M >= 2): every W steps a
// snapshot of X; after M + 1 snapshots x_0 .. x_M (differences u_a = x_{a+1}
// - x_a), per case the coefficients gamma minimising || sum_j gamma_j u_j ||
// with sum_j gamma_j = 1 (normal equations G y = 1 with a relative ridge of
// 1e-12, gamma = y / sum y), and X += sum_a c_a u_a with c_a = -sum_{j<=a}
// gamma_j, i.e. X = sum_j gamma_j x_j.  A case is left alone (c = 0) when its
// differences do not shrink (u_{M-1} no smaller than u_0: not yet in the
// contracting regime), when the solve is not finite, or when the step would
// exceed 500 times the last difference.  The new X is the first snapshot of
// the next cycle.
bool rre_solve(int m, const double* packed, double* c) {
    double G[kRreMaxOrder][kRreMaxOrder];
    int v = 0;
    for (int a = 0; a < m; ++a)
        for (int b = a; b < m; ++b) G[a][b] = G[b][a] = packed[v++];
    for (int a = 0; a < m; ++a) c[a] = 0.0;
    double tr = 0.0;
    for (int a = 0; a < m; ++a) tr += G[a][a];
    if (!(tr > 0.0) || !std::isfinite(tr)) return false;
    if (!(G[m - 1][m - 1] < G[0][0])) return false;
    double A[kRreMaxOrder][kRreMaxOrder];
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) A[a][b] = G[a][b] / tr + (a == b ? 1e-12 : 0.0);
    // Cholesky A = R^T R, then R^T R y = 1
    double R[kRreMaxOrder][kRreMaxOrder] = {};
    for (int i = 0; i < m; ++i) {
        for (int j = i; j < m; ++j) {
            double sum = A[i][j];
            for (int k = 0; k < i; ++k) sum -= R[k][i] * R[k][j];
            if (i == j) {
                if (!(sum > 0.0)) return false;
                R[i][i] = std::sqrt(sum);
            } else {
                R[i][j] = sum / R[i][i];
            }
        }
    }
    double y[kRreMaxOrder];
    for (int i = 0; i < m; ++i) {
        double sum = 1.0;
        for (int k = 0; k < i; ++k) sum -= R[k][i] * y[k];
        y[i] = sum / R[i][i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double sum = y[i];
        for (int k = i + 1; k < m; ++k) sum -= R[i][k] * y[k];
        y[i] = sum / R[i][i];
    }
    double sy = 0.0;
    for (int i = 0; i < m; ++i) sy += y[i];
    if (!(std::fabs(sy) > 0.0) || !std::isfinite(sy)) return false;
    double run = 0.0;
    for (int a = 0; a < m; ++a) {
        run += y[a] / sy;
        c[a] = -run;
    }
    // predicted step norm^2 = c^T G c
    double step = 0.0;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) step += c[a] * G[a][b] * c[b];
    if (!std::isfinite(step) || step > 500.0 * 500.0 * G[m - 1][m - 1]) {
        for (int a = 0; a < m; ++a) c[a] = 0.0;
        return false;
    }
    return true;
}

lbms_status rre_begin(lbms_ctx* c, Extrapolator& ex) {
    Launch& L = c->L;
    const int m = c->opt.extrapolate_modes;
    const int nv = m * (m + 1) / 2;
    if (!L.b.rre_ring) {
        // sized for the order of this handle's option (fixed at create)
        L.b.rre_ring = static_cast<double*>(dev_alloc(c, (size_t)(m + 1) * 3 * L.S * sizeof(double)));
        L.b.rre_partials = static_cast<double*>(dev_alloc(c, (size_t)L.n_segs * nv * sizeof(double)));
        L.b.rre_out = static_cast<double*>(dev_alloc(c, (size_t)L.n_cases * nv * sizeof(double)));
        L.b.rre_coef = static_cast<double*>(dev_alloc(c, (size_t)L.n_cases * m * sizeof(double)));
        if (!L.b.rre_ring || !L.b.rre_partials || !L.b.rre_out || !L.b.rre_coef)
            return fail(c, LBMS_ENOMEM, "reduced-rank extrapolation buffers");
    }
    ex.rre_coef.assign((size_t)L.n_cases * m, 0.0);
    ex.coef.assign(L.n_cases, 0.0);
    ex.polish.assign(L.n_cases, 0);
    ex.polish_n.assign(L.n_cases, 0);
    // the first snapshot of a cycle waits W / 8 steps, past the fast
    // transient that follows a start or a jump (it does not decay
    // geometrically and would corrupt the first difference)
    ex.rre_n = 0;
    ex.since = c->opt.extrapolate_every - std::max<int64_t>(1, c->opt.extrapolate_every / 8);
    return LBMS_OK;
}

// One snapshot; at the end of a cycle the extrapolation.  ex.coef[k] != 0
// marks the cases that moved.
lbms_status rre_check(lbms_ctx* c, Extrapolator& ex) {
    Launch& L = c->L;
    const int m = c->opt.extrapolate_modes;
    const int nv = m * (m + 1) / 2;
    const int n = L.n_cases;
    ex.since = 0;
    for (int k = 0; k < n; ++k) ex.coef[k] = 0.0;
    CK(launch_rre_snapshot(L, ex.rre_n, c->stream), "extrapolation snapshot");
    if (ex.rre_n++ == 0) return LBMS_OK;
    // a full cycle, or an early one (at least two differences) for the
    // final extrapolation of cases that met tol; an early cycle moves only
    // those cases
    bool pending = false;
    for (int k = 0; k < n; ++k) pending = pending || ex.polish[k] == 1;
    const bool full_cycle = ex.rre_n > m;
    if (!full_cycle && !(pending && ex.rre_n >= 3)) return LBMS_OK;
    const int mm = full_cycle ? m : ex.rre_n - 1;
    const int nvv = mm * (mm + 1) / 2;
    CK(launch_rre_gram(L, mm, c->stream), "extrapolation Gram matrices");
    std::vector<double> gram((size_t)n * nvv);
    CK(cudaMemcpyAsync(gram.data(), L.b.rre_out, gram.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "Gram readback");
    CK(cudaStreamSynchronize(c->stream), "Gram readback");
    c->d2h += gram.size() * sizeof(double);
    ex.rre_coef.assign((size_t)n * mm, 0.0);
    for (int k = 0; k < n; ++k) {
        if (!full_cycle && ex.polish[k] != 1) continue;
        if (rre_solve(mm, gram.data() + (size_t)k * nvv, ex.rre_coef.data() + (size_t)k * mm)) ex.coef[k] = 1.0;
        if (ex.polish[k] == 1) ex.polish[k] = 2;
    }
    CK(cudaMemcpyAsync(L.b.rre_coef, ex.rre_coef.data(), ex.rre_coef.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream),
       "extrapolation coefficients");
    c->h2d += ex.rre_coef.size() * sizeof(double);
    CK(launch_rre_apply(L, mm, c->stream), "extrapolation kernel");
    ex.rre_n = 0;
    ex.since = c->opt.extrapolate_every - std::max<int64_t>(1, c->opt.extrapolate_every / 8);
    return LBMS_OK;
}

}  // namespace

namespace lbms {

bool case_view(const lbms_ctx* c, int k, CaseView* v) {
    if (!c || k < 0 || k >= (int)c->cases.size() || !v) return false;
    const CaseHost& cs = c->cases[k];
    v->nx = cs.nx;
    v->ny = cs.ny;
    v->nz = cs.nz;
    v->N = cs.N;
    v->nf = cs.nf;
    v->fluid_cell = cs.fluid_cell.data();
    for (int s = 0; s < 3; ++s) v->x_in[s] = cs.x_in[s];
    v->current = cs.current;
    v->periodic_x = cs.periodic_x != 0;
    v->has_bc = cs.has_bc;
    return true;
}

bool case_profile_1d(const lbms_ctx* c, int k, std::vector<double>& prof) {
    if (!c || k < 0 || k >= (int)c->cases.size()) return false;
    const CaseHost& cs = c->cases[k];
    if (cs.periodic_x) return false;
    return profile_1d(c->gas, cs, cs.current, prof);
}

}  // namespace lbms

extern "C" {

void lbms_default_options(lbms_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = LBMS_FP32;
    o->coupling = LBMS_COUPLING_MS;
    o->tau_min = 1.0;
    o->tau_max = 5.0;
    o->dt_s = 0.0;
    o->check_every = 100;
    o->extrapolate_modes = 1;
}

const char* lbms_status_string(lbms_status s) {
    switch (s) {
        case LBMS_OK: return "ok";
        case LBMS_EINVAL: return "invalid argument";
        case LBMS_ENOMEM: return "out of memory";
        case LBMS_ECUDA: return "CUDA error";
        case LBMS_ENOTCONVERGED: return "not converged";
        case LBMS_EUNSTABLE: return "non-finite mole fractions";
        case LBMS_EDEPLETED: return "reactant depleted";
        case LBMS_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char* lbms_last_error(const lbms_ctx* c) { return c ? c->err.c_str() : t_create_error.c_str(); }

lbms_status lbms_create_batch(int n_cases, const lbms_geometry* geoms, const lbms_species* sp,
                              const lbms_diffusivities* df, double T_K, double p_Pa, const lbms_options* opt,
                              lbms_ctx** out) {
    if (!out) return LBMS_EINVAL;
    *out = nullptr;
    t_create_error.clear();
    lbms_ctx* c = new (std::nothrow) lbms_ctx();
    if (!c) return LBMS_ENOMEM;
    auto bail = [&](lbms_status s) {
        // the message stays readable through lbms_last_error(NULL) on this thread
        t_create_error = c->err;
        release(c);
        delete c;
        return s;
    };
    if (opt)
        c->opt = *opt;
    else
        lbms_default_options(&c->opt);
    if (c->opt.check_every <= 0) c->opt.check_every = 100;
    if (c->opt.extrapolate_every < 0) c->opt.extrapolate_every = 0;
    if (c->opt.extrapolate_modes < 0 || c->opt.extrapolate_modes > kRreMaxOrder)
        return bail(fail(c, LBMS_EINVAL, "extrapolate_modes must be in 0..%d", kRreMaxOrder));
    if (c->opt.step_variant < 0 || c->opt.step_variant > kStepVariants) return bail(fail(c, LBMS_EINVAL, "step_variant out of range"));
    if (c->opt.init_mode != LBMS_INIT_UNIFORM && c->opt.init_mode != LBMS_INIT_PROFILE_1D)
        return bail(fail(c, LBMS_EINVAL, "init_mode must be LBMS_INIT_UNIFORM or LBMS_INIT_PROFILE_1D"));
    if (c->opt.outlet_bc != LBMS_OUTLET_FLUX && c->opt.outlet_bc != LBMS_OUTLET_EXTRAPOLATED)
        return bail(fail(c, LBMS_EINVAL, "outlet_bc must be LBMS_OUTLET_FLUX or LBMS_OUTLET_EXTRAPOLATED"));
    if (c->opt.grad_stencil != LBMS_GRAD_CENTRAL && c->opt.grad_stencil != LBMS_GRAD_FORWARD)
        return bail(fail(c, LBMS_EINVAL, "grad_stencil must be LBMS_GRAD_CENTRAL or LBMS_GRAD_FORWARD"));
    if (c->opt.outlet_bc == LBMS_OUTLET_EXTRAPOLATED && c->opt.step_variant > 0 &&
        !kVariantPerCell[c->opt.step_variant - 1])
        return bail(fail(c, LBMS_EINVAL, "the extrapolated outlet needs a per-cell step variant (7 to 10)"));
    if (n_cases < 1) return bail(fail(c, LBMS_EINVAL, "n_cases must be >= 1"));
    if (!geoms) return bail(fail(c, LBMS_EINVAL, "geometry is NULL"));
    if (!sp) return bail(fail(c, LBMS_EINVAL, "species is NULL"));
    const int dim = geoms[0].dim;
    if (dim != 2 && dim != 3) return bail(fail(c, LBMS_EINVAL, "dim must be 2 or 3"));
    for (int k = 0; k < n_cases; ++k) {
        const lbms_geometry* g = &geoms[k];
        if (g->dim != dim) return bail(fail(c, LBMS_EINVAL, "case %d: every case of a batch needs the same dim", k));
        if (g->nx < 1 || g->ny < 1 || g->nz < 1) return bail(fail(c, LBMS_EINVAL, "case %d: nx, ny, nz must be >= 1", k));
        if (dim == 2 && g->nz != 1) return bail(fail(c, LBMS_EINVAL, "case %d: nz must be 1 when dim = 2", k));
        if (!g->periodic_x && g->nx < 3)
            return bail(fail(c, LBMS_EINVAL, "case %d: nx must be >= 3 with an inlet and outlet", k));
        if (!g->solid) return bail(fail(c, LBMS_EINVAL, "case %d: solid mask is NULL", k));
        if (!(g->length_x_m > 0.0) || !std::isfinite(g->length_x_m))
            return bail(fail(c, LBMS_EINVAL, "case %d: length_x_m must be finite and > 0", k));
    }
    if (sp->n != 3) return bail(fail(c, LBMS_EINVAL, "only ternary mixtures (n = 3) are supported"));
    if (!sp->stoich || sp->electrons <= 0) return bail(fail(c, LBMS_EINVAL, "stoich and electrons > 0 are required"));
    if ((!df || !df->D_binary_m2s || (df->pore_diameter_m > 0.0)) && !sp->molar_mass)
        return bail(fail(c, LBMS_EINVAL, "molar_mass is required"));
    if ((!df || !df->D_binary_m2s) && !sp->fuller_volume)
        return bail(fail(c, LBMS_EINVAL, "fuller_volume is required without D_binary_m2s"));
    if (sp->molar_mass)
        for (int i = 0; i < 3; ++i)
            if (!(sp->molar_mass[i] > 0.0)) return bail(fail(c, LBMS_EINVAL, "molar_mass must be > 0"));
    if (!(T_K > 0.0) || !(p_Pa > 0.0) || !std::isfinite(T_K) || !std::isfinite(p_Pa))
        return bail(fail(c, LBMS_EINVAL, "T and p must be finite and > 0"));
    if (c->opt.precision != LBMS_FP64 && c->opt.precision != LBMS_FP32 && c->opt.precision != LBMS_FP16)
        return bail(fail(c, LBMS_EINVAL, "precision must be LBMS_FP64, LBMS_FP32 or LBMS_FP16"));
    if (!(c->opt.tau_min > 0.5) || !(c->opt.tau_max >= c->opt.tau_min))
        return bail(fail(c, LBMS_EINVAL, "need 0.5 < tau_min <= tau_max"));
    if (c->opt.coupling != LBMS_COUPLING_MS && c->opt.coupling != LBMS_COUPLING_TAU_ONLY)
        return bail(fail(c, LBMS_EINVAL, "unknown coupling"));

    c->dim = dim;
    c->Q = dim == 2 ? D2Q9::Q : D3Q19::Q;
    c->stream = static_cast<cudaStream_t>(c->opt.stream);

    // fluid cells and boundary rows of every case, laid out one after another
    c->cases.resize(n_cases);
    std::vector<std::vector<int>> index_of(n_cases);
    std::vector<int> rows_x0, rows_x1, rows_out;
    int64_t next = 0;
    for (int k = 0; k < n_cases; ++k) {
        const lbms_geometry* g = &geoms[k];
        CaseHost& cs = c->cases[k];
        cs.nx = g->nx;
        cs.ny = g->ny;
        cs.nz = g->nz;
        cs.periodic_x = g->periodic_x ? 1 : 0;
        cs.length_x = g->length_x_m;
        cs.N = (int64_t)cs.nx * cs.ny * cs.nz;
        index_of[k].assign((size_t)cs.N, -1);
        for (int64_t cell = 0; cell < cs.N; ++cell) {
            if (g->solid[cell]) continue;
            index_of[k][cell] = (int)cs.fluid_cell.size();
            cs.fluid_cell.push_back(cell);
        }
        if (cs.fluid_cell.empty()) return bail(fail(c, LBMS_EINVAL, "case %d: the mask has no fluid cell", k));
        cs.nf = (int)cs.fluid_cell.size();
        cs.base = (int)next;
        next += ((int64_t)cs.nf + kCaseAlign - 1) / kCaseAlign * kCaseAlign;
        // cell indices are 32-bit; the per-species offsets (link x row stride)
        // are bounded by the Q x stride check below
        if (next >= (int64_t)std::numeric_limits<int>::max() - kCaseAlign)
            return bail(fail(c, LBMS_EINVAL, "too many fluid cells for 32-bit indices"));
        cs.row_first = (int)rows_x0.size();
        cs.nrows = cs.ny * cs.nz;
        for (int r = 0; r < cs.nrows; ++r) {
            const int64_t b = (int64_t)r * cs.nx;
            const int i0 = index_of[k][b], i1 = cs.nx > 1 ? index_of[k][b + 1] : -1, io = index_of[k][b + cs.nx - 1];
            if (!cs.periodic_x && (i0 < 0 || io < 0))
                return bail(fail(c, LBMS_EINVAL, "case %d: inlet (x = 0) and outlet (x = nx-1) columns must be fluid", k));
            rows_x0.push_back(i0 >= 0 ? cs.base + i0 : -1);
            rows_x1.push_back(i1 >= 0 ? cs.base + i1 : -1);
            rows_out.push_back(io >= 0 ? cs.base + io : -1);
        }
    }
    lbms_status st = compute_props(c, sp, df, T_K, p_Pa);
    if (st != LBMS_OK) return bail(st);

    Launch& L = c->L;
    L.dim = dim;
    L.precision = c->opt.precision;
    L.n_cases = n_cases;
    L.ncells = (int)next;
    L.S = ((int64_t)L.ncells + 31) / 32 * 32;
    L.total_rows = (int)rows_x0.size();
    if ((int64_t)c->Q * L.S >= (int64_t)std::numeric_limits<int>::max())
        return bail(fail(c, LBMS_EINVAL, "too many fluid cells: Q x cells must stay below 2^31"));
    L.D12 = c->gas.D_lat[0][1];
    L.D13 = c->gas.D_lat[0][2];
    L.D23 = c->gas.D_lat[1][2];
    for (int s = 0; s < 3; ++s) L.stoich[s] = c->gas.stoich[s];
    L.tau_min = c->opt.tau_min;
    L.tau_max = c->opt.tau_max;
    L.drift = c->opt.coupling == LBMS_COUPLING_MS ? 1 : 0;
    L.grad_forward = c->opt.grad_stencil == LBMS_GRAD_FORWARD ? 1 : 0;
    L.outlet_extrap = c->opt.outlet_bc == LBMS_OUTLET_EXTRAPOLATED ? 1 : 0;

    // reduction segments and block -> case tables
    std::vector<int2> segs, case_segs(n_cases), case_rows(n_cases);
    std::vector<int> seg_case;
    for (int k = 0; k < n_cases; ++k) {
        const CaseHost& cs = c->cases[k];
        case_segs[k] = make_int2((int)segs.size(), 0);
        for (int j = 0; j < cs.nf; j += kSegCells) {
            segs.push_back(make_int2(cs.base + j, std::min(kSegCells, cs.nf - j)));
            seg_case.push_back(k);
        }
        case_segs[k].y = (int)segs.size() - case_segs[k].x;
        case_rows[k] = make_int2(cs.row_first, cs.nrows);
    }
    L.n_segs = (int)segs.size();
    std::vector<std::vector<int>> blk_case(kStepVariants);
    for (int v = 0; v < kStepVariants; ++v) {
        const int W = kVariantCells[v];
        L.nblk[v] = L.ncells / W;
        blk_case[v].resize(L.nblk[v]);
        int k = 0;
        for (int b = 0; b < L.nblk[v]; ++b) {
            while (k + 1 < n_cases && b * W >= c->cases[k + 1].base) ++k;
            blk_case[v][b] = k;
        }
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
    int smc = 0;
    if (cudaDeviceGetAttribute(&smc, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && smc > 0) L.sm_count = smc;
    e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "create capture stream"));
    e = cudaMallocHost(&c->host_out, (size_t)n_cases * kCaseOutSlots * sizeof(double));
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "pinned readback buffer"));

    const int nbw = dim == 2 ? nb_width<D2Q9>() : nb_width<D3Q19>();
    const size_t fbytes = (size_t)3 * c->Q * L.S * pop_size(L.precision);
    const size_t xbytes = (size_t)3 * L.S * x_size(L.precision);
    const size_t sbytes = (size_t)3 * L.S * sizeof(double);
    const size_t cbytes = (size_t)n_cases * case_bc_size(L.precision);
    for (int k = 0; k < 2; ++k) {
        L.b.f[k] = dev_alloc(c, fbytes);
        L.b.X[k] = dev_alloc(c, xbytes);
    }
    L.b.snap = static_cast<double*>(dev_alloc(c, sbytes));
    L.b.nbr = static_cast<int*>(dev_alloc(c, (size_t)nbw * L.S * sizeof(int)));
    L.b.rows = static_cast<int*>(dev_alloc(c, 3 * (size_t)L.total_rows * sizeof(int)));
    L.b.case_rows = static_cast<int2*>(dev_alloc(c, (size_t)n_cases * sizeof(int2)));
    L.b.cases = dev_alloc(c, cbytes);
    for (int v = 0; v < kStepVariants; ++v) L.b.blk_case[v] = static_cast<int*>(dev_alloc(c, (size_t)L.nblk[v] * sizeof(int)));
    L.b.segs = static_cast<int2*>(dev_alloc(c, segs.size() * sizeof(int2)));
    L.b.case_segs = static_cast<int2*>(dev_alloc(c, (size_t)n_cases * sizeof(int2)));
    L.b.seg_case = static_cast<int*>(dev_alloc(c, seg_case.size() * sizeof(int)));
    L.b.coef = static_cast<double*>(dev_alloc(c, (size_t)n_cases * sizeof(double)));
    L.b.partials = static_cast<double*>(dev_alloc(c, segs.size() * 10 * sizeof(double)));
    L.b.case_out = static_cast<double*>(dev_alloc(c, (size_t)n_cases * kCaseOutSlots * sizeof(double)));
    bool ok = L.b.f[0] && L.b.f[1] && L.b.X[0] && L.b.X[1] && L.b.snap && L.b.nbr && L.b.rows && L.b.case_rows &&
              L.b.cases && L.b.segs && L.b.case_segs && L.b.seg_case && L.b.coef && L.b.partials && L.b.case_out;
    for (int v = 0; v < kStepVariants; ++v) ok = ok && L.b.blk_case[v];
    if (!ok) return bail(fail(c, LBMS_ENOMEM, "device allocation of %zu bytes failed", 2 * fbytes + 2 * xbytes + sbytes));

    // Neighbour tables, built on the device from each case's dense
    // fluid-index map.  The 16-bit offset table is kept when the links
    // whose offsets do not fit (periodic wraps) are rare, at most 1 in 16;
    // those are marked NB16_FAR and read the 32-bit table.
    const int nbw16 = dim == 2 ? nb16_width<D2Q9>() : nb16_width<D3Q19>();
    {
        int64_t max_n = 1, max_nf = 1;
        for (const auto& cs : c->cases) {
            max_n = std::max<int64_t>(max_n, cs.N);
            max_nf = std::max<int64_t>(max_nf, cs.nf);
        }
        int16_t* nb16 = static_cast<int16_t*>(dev_alloc(c, (size_t)nbw16 * L.S * sizeof(int16_t)));
        int* d_index = static_cast<int*>(dev_alloc(c, (size_t)max_n * sizeof(int)));
        int64_t* d_cells = static_cast<int64_t*>(dev_alloc(c, (size_t)max_nf * sizeof(int64_t)));
        unsigned long long* d_counts = static_cast<unsigned long long*>(dev_alloc(c, 2 * sizeof(unsigned long long)));
        if (!d_index || !d_cells || !d_counts)
            return bail(fail(c, LBMS_ENOMEM, "device allocation for the neighbour tables failed"));
        e = cudaMemsetAsync(L.b.nbr, 0xFF, (size_t)nbw * L.S * sizeof(int), c->stream);   // NB_SOLID
        if (e == cudaSuccess && nb16) e = launch_fill16(nb16, (int64_t)nbw16 * L.S, (int16_t)NB16_SOLID, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_counts, 0, 2 * sizeof(unsigned long long), c->stream);
        for (int k = 0; k < n_cases && e == cudaSuccess; ++k) {
            const CaseHost& cs = c->cases[k];
            e = cudaMemcpyAsync(d_index, index_of[k].data(), (size_t)cs.N * sizeof(int), cudaMemcpyHostToDevice,
                                c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_cells, cs.fluid_cell.data(), (size_t)cs.nf * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = launch_build_neighbours(dim, d_cells, d_index, cs.nf, cs.base, cs.nx, cs.ny, cs.nz, cs.periodic_x,
                                            L.b.nbr, nb16, d_counts, c->stream);
            // the host maps are reused by the next case's copies: wait for this one
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            c->h2d += (size_t)cs.N * sizeof(int) + (size_t)cs.nf * sizeof(int64_t);
        }
        unsigned long long counts[2] = {0, 0};
        if (e == cudaSuccess)
            e = cudaMemcpy(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "building the neighbour tables"));
        dev_free(c, d_index);
        dev_free(c, d_cells);
        dev_free(c, d_counts);
        if (nb16 && counts[1] * 16 <= counts[0])
            L.b.nbr16 = nb16;
        else if (nb16)
            dev_free(c, nb16);
    }
    // Row-bitmask decode (kNbRowMask variants): a coordinate word per cell
    // and, per case, (y, z) row and 32-voxel word w, a 64-bit window of the
    // fluid flags of voxels 32 w - 16 .. 32 w + 47 and the fluid index of the
    // first fluid voxel at or after 32 w - 16.  Built on the host from the
    // fluid-index maps; not built when a case is periodic in x or too large
    // for the coordinate word.
    {
        bool ok_rm = true;
        int64_t entries = 0;
        for (const auto& cs : c->cases) {
            ok_rm = ok_rm && !cs.periodic_x && cs.nx <= kRowMaskMaxNx && cs.ny <= kRowMaskMaxNy &&
                    cs.nz <= kRowMaskMaxNz;
            entries += (int64_t)cs.ny * cs.nz * ((cs.nx + 31) / 32);
        }
        ok_rm = ok_rm && entries < (int64_t)std::numeric_limits<int>::max();
        if (ok_rm) {
            std::vector<uint32_t> code((size_t)L.S, 0xFFFFFFFFu);
            std::vector<uint4> tab((size_t)entries);
            int64_t next_tab = 0;
            for (int k = 0; k < n_cases; ++k) {
                CaseHost& cs = c->cases[k];
                cs.wpr = (cs.nx + 31) / 32;
                cs.tab = (int)next_tab;
                next_tab += (int64_t)cs.ny * cs.nz * cs.wpr;
                for (int li = 0; li < cs.nf; ++li) {
                    const int64_t cell = cs.fluid_cell[li];
                    const uint32_t x = (uint32_t)(cell % cs.nx);
                    const uint32_t y = (uint32_t)((cell / cs.nx) % cs.ny);
                    const uint32_t z = (uint32_t)(cell / ((int64_t)cs.nx * cs.ny));
                    code[(size_t)cs.base + li] = x | (y << 11) | (z << 21);
                }
                std::vector<uint32_t> words((size_t)cs.wpr + 2);   // words[m + 1] = voxels 32 m .. 32 m + 31
                int count = cs.base;                                // fluid index of the next fluid voxel
                for (int r = 0; r < cs.ny * cs.nz; ++r) {
                    std::fill(words.begin(), words.end(), 0u);
                    const int* row = index_of[k].data() + (int64_t)r * cs.nx;
                    for (int x = 0; x < cs.nx; ++x)
                        if (row[x] >= 0) words[(size_t)(x >> 5) + 1] |= 1u << (x & 31);
                    for (int w = 0; w < cs.wpr; ++w) {
                        const uint64_t win = (uint64_t)(words[w] >> 16) | ((uint64_t)words[w + 1] << 16) |
                                             ((uint64_t)(words[w + 2] & 0xFFFFu) << 48);
                        // count = index of the first fluid voxel at or after 32 w; the
                        // window starts 16 voxels earlier
                        const int before = count - __builtin_popcount(words[w] >> 16);
                        tab[(size_t)cs.tab + (size_t)r * cs.wpr + w] =
                            make_uint4((uint32_t)win, (uint32_t)(win >> 32), (uint32_t)before, 0u);
                        count += __builtin_popcount(words[w + 1]);
                    }
                }
                if (count != cs.base + cs.nf) return bail(fail(c, LBMS_EINVAL, "case %d: row table count mismatch", k));
            }
            L.b.cell_code = static_cast<uint32_t*>(dev_alloc(c, (size_t)L.S * sizeof(uint32_t)));
            L.b.rowtab = static_cast<uint4*>(dev_alloc(c, (size_t)std::max<int64_t>(entries, 1) * sizeof(uint4)));
            if (!L.b.cell_code || !L.b.rowtab) return bail(fail(c, LBMS_ENOMEM, "row-bitmask tables"));
            e = cudaMemcpyAsync(L.b.cell_code, code.data(), code.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                c->stream);
            if (e == cudaSuccess && entries)
                e = cudaMemcpyAsync(L.b.rowtab, tab.data(), tab.size() * sizeof(uint4), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return bail(cuda_fail(c, e, "upload of the row-bitmask tables"));
            c->h2d += code.size() * sizeof(uint32_t) + tab.size() * sizeof(uint4);
        }
    }
    std::vector<int> rows;
    rows.reserve(3 * rows_x0.size());
    rows.insert(rows.end(), rows_x0.begin(), rows_x0.end());
    rows.insert(rows.end(), rows_x1.begin(), rows_x1.end());
    rows.insert(rows.end(), rows_out.begin(), rows_out.end());
    c->case_bc.assign(cbytes, 0);
    auto up = [&](void* dst, const void* src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->stream);
        c->h2d += n;
    };
    up(L.b.rows, rows.data(), rows.size() * sizeof(int));
    up(L.b.case_rows, case_rows.data(), case_rows.size() * sizeof(int2));
    up(L.b.segs, segs.data(), segs.size() * sizeof(int2));
    up(L.b.case_segs, case_segs.data(), case_segs.size() * sizeof(int2));
    up(L.b.seg_case, seg_case.data(), seg_case.size() * sizeof(int));
    for (int v = 0; v < kStepVariants; ++v) up(L.b.blk_case[v], blk_case[v].data(), blk_case[v].size() * sizeof(int));
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(L.b.f[k], 0, fbytes, c->stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(L.b.X[k], 0, xbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.b.snap, 0, sbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.b.cases, 0, cbytes, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "upload of the neighbour table"));
    for (int k = 0; k < n_cases && st == LBMS_OK; ++k) st = upload_case_bc(c, k);
    if (st != LBMS_OK) return bail(st);
    *out = c;
    return LBMS_OK;
}

lbms_status lbms_create(const lbms_geometry* geom, const lbms_species* sp, const lbms_diffusivities* df, double T_K,
                        double p_Pa, const lbms_options* opt, lbms_ctx** out) {
    if (!geom) {
        if (out) *out = nullptr;
        t_create_error = "geometry is NULL";
        return LBMS_EINVAL;
    }
    return lbms_create_batch(1, geom, sp, df, T_K, p_Pa, opt, out);
}

lbms_status lbms_set_bc(lbms_ctx* c, const double* x_inlet, double current_A_cm2) {
    if (!c || c->allocs.empty()) return fail(c, LBMS_ESTATE, "handle has no device state");
    for (int k = 0; k < (int)c->cases.size(); ++k) {
        lbms_status st = set_case_bc(c, k, x_inlet, current_A_cm2);
        if (st != LBMS_OK) return st;
    }
    return LBMS_OK;
}

lbms_status lbms_batch_set_bc(lbms_ctx* c, int k, const double* x_inlet, double current_A_cm2) {
    if (!c || c->allocs.empty()) return fail(c, LBMS_ESTATE, "handle has no device state");
    if (bad_case(c, k)) return fail(c, LBMS_EINVAL, "case index %d out of range", k);
    return set_case_bc(c, k, x_inlet, current_A_cm2);
}

lbms_status lbms_batch_set_fields(lbms_ctx* c, int k, const double* X) {
    if (!c || c->allocs.empty()) return fail(c, LBMS_ESTATE, "handle has no device state");
    if (bad_case(c, k)) return fail(c, LBMS_EINVAL, "case index %d out of range", k);
    if (!c->cases[k].has_bc) return fail(c, LBMS_ESTATE, "set the boundary data of case %d first", k);
    if (!X) return fail(c, LBMS_EINVAL, "X is NULL");
    lbms_status st = upload_field(c, k, X);
    if (st == LBMS_OK) c->steps = 0;
    return st;
}

lbms_status lbms_set_fields(lbms_ctx* c, const double* X) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc before lbms_set_fields");
    return lbms_batch_set_fields(c, 0, X);
}

lbms_status lbms_step(lbms_ctx* c, int64_t nsteps) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "set the boundary data of every case first");
    if (nsteps < 0) return fail(c, LBMS_EINVAL, "nsteps must be >= 0");
    return launch_steps(c, nsteps);
}

lbms_status lbms_batch_residuals(lbms_ctx* c, int K, double* residuals) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "set the boundary data of every case first");
    if (K < 1 || !residuals) return fail(c, LBMS_EINVAL, "need K >= 1 and a residual array");
    return case_residuals(c, K, residuals);
}

lbms_status lbms_residual(lbms_ctx* c, int K, double* residual) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (K < 1 || !residual) return fail(c, LBMS_EINVAL, "need K >= 1 and a residual pointer");
    std::vector<double> r(c->cases.size());
    lbms_status st = case_residuals(c, K, r.data());
    double m = 0.0;
    for (double v : r) m = std::max(m, v);
    *residual = st == LBMS_EUNSTABLE ? std::numeric_limits<double>::infinity() : m;
    return st;
}

lbms_status lbms_batch_run_to_residual(lbms_ctx* c, double tol, int64_t max_steps, int64_t* steps_taken,
                                       int64_t* case_steps, double* final_residuals) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "set the boundary data of every case first");
    if (!(tol >= 0.0) || max_steps < 0) return fail(c, LBMS_EINVAL, "need tol >= 0 and max_steps >= 0");
    const int n = (int)c->cases.size();
    const int K = c->opt.check_every;
    std::vector<double> r(n, std::numeric_limits<double>::infinity());
    std::vector<int64_t> met(n, -1);
    int64_t done = 0;
    CK(launch_case_residuals(c->L, 1, c->stream), "residual kernels");  // snapshots start here
    lbms_status st = LBMS_OK;
    const int64_t W = c->opt.extrapolate_every;
    const bool rre = c->opt.extrapolate_modes >= 2;
    Extrapolator ex;
    if (W > 0) st = rre ? rre_begin(c, ex) : extrap_begin(c, ex);
    bool all = false;
    while (st == LBMS_OK && done < max_steps && !all) {
        const int64_t k = std::min<int64_t>(K, max_steps - done);
        st = launch_steps(c, k);
        if (st != LBMS_OK) break;
        done += k;
        st = case_residuals(c, (int)k, r.data());
        if (st != LBMS_OK) break;
        if (W > 0 && (ex.since += k) >= W) {
            st = rre ? rre_check(c, ex) : extrap_check(c, ex);
            if (st != LBMS_OK) break;
            // a jump is never the last thing before a convergence decision:
            // the next residual check sees it in its K-step change
            bool any = false;
            for (double cf : ex.coef) any = any || cf != 0.0;
            if (any) continue;
        }
        all = true;
        for (int q = 0; q < n; ++q) {
            if (met[q] < 0 && r[q] <= tol) {
                // with extrapolation a case is done when it meets tol again
                // after one final extrapolation taken at its next W-step check
                if (W > 0 && ex.polish[q] == 0)
                    ex.polish[q] = 1;
                else if (W <= 0 || ex.polish[q] == 2)
                    met[q] = done;
            }
            all = all && met[q] >= 0;
        }
    }
    if (steps_taken) *steps_taken = done;
    if (case_steps)
        for (int q = 0; q < n; ++q) case_steps[q] = met[q];
    if (final_residuals)
        for (int q = 0; q < n; ++q) final_residuals[q] = r[q];
    if (st != LBMS_OK) return st;
    if (!all) return fail(c, LBMS_ENOTCONVERGED, "not every case reached %.3e after %lld steps", tol, (long long)done);
    return LBMS_OK;
}

lbms_status lbms_run_to_residual(lbms_ctx* c, double tol, int64_t max_steps, int64_t* steps_taken,
                                 double* final_residual) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    std::vector<double> r(c->cases.size());
    lbms_status st = lbms_batch_run_to_residual(c, tol, max_steps, steps_taken, nullptr, r.data());
    if (final_residual) {
        double m = 0.0;
        for (double v : r) m = std::max(m, v);
        *final_residual = m;
    }
    return st;
}

lbms_status lbms_batch_get_fields(lbms_ctx* c, int k, double* X, double* u, double* tau) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "set the boundary data of every case first");
    if (bad_case(c, k)) return fail(c, LBMS_EINVAL, "case index %d out of range", k);
    const CaseHost& cs = c->cases[k];
    const int64_t S = c->L.S;
    const int prec = c->L.precision;
    if (X) {
        const int rows = x_rows(prec);
        const size_t word = x_word(prec);
        std::vector<unsigned char> b((size_t)rows * cs.nf * word);
        const unsigned char* src = static_cast<const unsigned char*>(c->L.b.X[c->L.cur]) + (size_t)cs.base * word;
        CK(cudaMemcpy2DAsync(b.data(), cs.nf * word, src, S * word, cs.nf * word, rows, cudaMemcpyDeviceToHost, c->stream),
           "read X");
        CK(cudaStreamSynchronize(c->stream), "read X");
        c->d2h += b.size();
        std::fill(X, X + 3 * cs.N, 0.0);
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i < cs.nf; ++i) X[s * cs.N + cs.fluid_cell[i]] = get_x(prec, b.data(), cs.nf, (int64_t)s * cs.nf + i);
    }
    if (u || tau) {
        const size_t es = field_size(prec);
        const int rows = 3 + 3 * c->dim;
        if (!c->L.b.fields) {
            c->L.b.fields = dev_alloc(c, (size_t)rows * S * es);
            if (!c->L.b.fields) return fail(c, LBMS_ENOMEM, "fields buffer");
        }
        CK(launch_fields(c->L, c->stream), "fields kernel");
        std::vector<unsigned char> b((size_t)rows * cs.nf * es);
        const unsigned char* src = static_cast<const unsigned char*>(c->L.b.fields) + (size_t)cs.base * es;
        CK(cudaMemcpy2DAsync(b.data(), cs.nf * es, src, S * es, cs.nf * es, rows, cudaMemcpyDeviceToHost, c->stream),
           "read fields");
        CK(cudaStreamSynchronize(c->stream), "read fields");
        c->d2h += b.size();
        auto val = [&](int row, int i) {
            const size_t idx = (size_t)row * cs.nf + i;
            return prec == LBMS_FP64 ? reinterpret_cast<const double*>(b.data())[idx]
                                     : (double)reinterpret_cast<const float*>(b.data())[idx];
        };
        if (tau) {
            std::fill(tau, tau + 3 * cs.N, 0.0);
            for (int s = 0; s < 3; ++s)
                for (int i = 0; i < cs.nf; ++i) tau[s * cs.N + cs.fluid_cell[i]] = val(s, i);
        }
        if (u) {
            const double scale = cs.dx / cs.dt;
            std::fill(u, u + 3 * (size_t)c->dim * cs.N, 0.0);
            for (int s = 0; s < 3; ++s)
                for (int d = 0; d < c->dim; ++d)
                    for (int i = 0; i < cs.nf; ++i)
                        u[(s * c->dim + d) * cs.N + cs.fluid_cell[i]] = scale * val(3 + s * c->dim + d, i);
        }
    }
    return LBMS_OK;
}

lbms_status lbms_get_fields(lbms_ctx* c, double* X, double* u, double* tau) {
    return lbms_batch_get_fields(c, 0, X, u, tau);
}

lbms_status lbms_batch_overpotentials(lbms_ctx* c, double* eta_V, double* x_out_mean) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "set the boundary data of every case first");
    if (!eta_V) return fail(c, LBMS_EINVAL, "eta_V is NULL");
    lbms_status st = case_boundary(c);
    if (st != LBMS_OK) return st;
    lbms_status worst = LBMS_OK;
    for (int k = 0; k < (int)c->cases.size(); ++k) {
        if (c->cases[k].periodic_x) {
            eta_V[k] = std::numeric_limits<double>::quiet_NaN();
            worst = fail(c, LBMS_EINVAL, "case %d is periodic in x and has no outlet", k);
            continue;
        }
        st = overpotential_of(c, k, eta_V + k, x_out_mean ? x_out_mean + 3 * k : nullptr);
        if (st != LBMS_OK) worst = st;
    }
    return worst;
}

lbms_status lbms_overpotential(lbms_ctx* c, double* eta_V, double* x_out_mean) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (c->cases[0].periodic_x) return fail(c, LBMS_EINVAL, "a box periodic in x has no outlet");
    lbms_status st = case_boundary(c);
    if (st != LBMS_OK) return st;
    return overpotential_of(c, 0, eta_V, x_out_mean);
}

lbms_status lbms_boundary_flux(lbms_ctx* c, double* inlet_flux, double* totals) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (inlet_flux) {
        lbms_status st = case_boundary(c);
        if (st != LBMS_OK) return st;
        const double* o = c->host_out + (size_t)c->L.n_cases * 10;
        for (int s = 0; s < 3; ++s) inlet_flux[s] = o[s];
    }
    if (totals) {
        CK(launch_case_residuals(c->L, 0, c->stream), "sum kernels");
        lbms_status st = read_case_out(c, 0, (size_t)c->L.n_cases * 10);
        if (st != LBMS_OK) return st;
        for (int s = 0; s < 3; ++s) totals[s] = c->host_out[6 + s];
    }
    return LBMS_OK;
}

lbms_status lbms_get_info(const lbms_ctx* c, lbms_info* info) {
    if (!c || !info) return LBMS_EINVAL;
    std::memset(info, 0, sizeof(*info));
    const CaseHost& c0 = c->cases[0];
    for (const auto& cs : c->cases) {
        info->n_cells += cs.N;
        info->n_fluid += cs.nf;
    }
    info->q = c->Q;
    info->precision = c->opt.precision;
    info->dx_m = c0.dx;
    info->dt_s = c0.dt;
    info->C_t = c->gas.C_t;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            info->D_eff_m2s[i * 3 + j] = c->gas.D_eff[i][j];
            info->D_lat[i * 3 + j] = c->gas.D_lat[i][j];
        }
    for (int s = 0; s < 3; ++s) {
        info->q_lat[s] = c0.q[s];
        info->x_in[s] = c0.x_in[s];
    }
    info->current_A_cm2 = c0.current;
    info->steps = c->steps;
    info->device_bytes = c->device_bytes;
    info->h2d_bytes = c->h2d;
    info->d2h_bytes = c->d2h;
    info->n_cases = (int)c->cases.size();
    info->tile_cells = kVariantCells[c->L.variant];
    info->tile_min_blocks = kVariantMinBlocks[c->L.variant];
    info->neighbour_bits = kVariantNb[c->L.variant] == kNbOffset16 ? 16 : (kVariantNb[c->L.variant] == kNbRowMask ? 1 : 32);
    info->threads_per_cell = kVariantPerCell[c->L.variant] ? 1 : 3;
    return LBMS_OK;
}

lbms_status lbms_synchronize(lbms_ctx* c) {
    if (!c) return LBMS_EINVAL;
    CK(cudaStreamSynchronize(c->stream), "synchronize");
    return LBMS_OK;
}

void lbms_destroy(lbms_ctx* c) {
    if (!c) return;
    release(c);
    delete c;
}

}  // extern "C"
