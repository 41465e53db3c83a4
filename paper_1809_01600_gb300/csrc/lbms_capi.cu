// C ABI of the solver (declared in include/lbms.h): validation, host
// properties, fluid-cell indexing, device state, CUDA-graph stepping,
// residual loop and the FP64 post-processing of Eq. 43.
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
#include "lbms_lattice.cuh"
#include "lbms_props.cuh"

using namespace lbms;

struct lbms_ctx {
    // geometry
    int dim = 2, nx = 0, ny = 0, nz = 0, Q = 9, periodic_x = 0;
    int64_t N = 0;
    double length_x = 0.0;
    std::vector<int64_t> fluid_cell;  // dense index of each fluid cell, x-fastest order
    // properties and options
    GasProps gas{};
    lbms_options opt{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    // device state
    Launch L;
    std::vector<std::pair<void*, size_t>> allocs;
    size_t device_bytes = 0;
    double* host_red = nullptr;  // pinned, 2 * kRedSlots doubles
    uint64_t h2d = 0, d2h = 0;   // bytes copied across PCIe/C2C so far
    bool initialized = false;
    int64_t steps = 0;
    double x_in[3] = {0, 0, 0};
    double current = 0.0;
    // CUDA graphs of kGraphSteps steps, one per starting lattice parity
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
    if (c->host_red) cudaFreeHost(c->host_red);
    c->host_red = nullptr;
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->cap_stream = nullptr;
}

// Eqs. 40-42, C_t and the lattice scaling (dx, dt, D*).
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
    g.dx = c->periodic_x ? c->length_x / c->nx : c->length_x / (c->nx - 1);
    g.dt = c->opt.dt_s > 0.0 ? c->opt.dt_s : g.dx * g.dx / (6.0 * dmin);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) g.D_lat[i][j] = g.D_eff[i][j] * g.dt / (g.dx * g.dx);
    return LBMS_OK;
}

// Pull-neighbour table: row i holds, for k = 1..Q-1, the fluid index of the
// source x - e_k or an NB_* code, padded to nb_width ints.
template <class Lat>
void build_neighbours(const lbms_ctx* c, const std::vector<int>& index_of, int64_t S, std::vector<int>& nbr) {
    const int nf = (int)c->fluid_cell.size();
    constexpr int NW = nb_width<Lat>();
    nbr.assign((size_t)NW * S, NB_SOLID);
    for (int i = 0; i < nf; ++i) {
        const int64_t cell = c->fluid_cell[i];
        const int x = (int)(cell % c->nx);
        const int y = (int)((cell / c->nx) % c->ny);
        const int z = (int)(cell / ((int64_t)c->nx * c->ny));
        for (int k = 1; k < Lat::Q; ++k) {
            int sx = x - Lat::e(k, 0);
            const int sy = ((y - Lat::e(k, 1)) % c->ny + c->ny) % c->ny;
            const int sz = ((z - Lat::e(k, 2)) % c->nz + c->nz) % c->nz;
            int code;
            if (!c->periodic_x && sx < 0) {
                code = NB_INLET;
            } else if (!c->periodic_x && sx >= c->nx) {
                code = NB_OUTLET;
            } else {
                sx = (sx % c->nx + c->nx) % c->nx;
                const int j = index_of[((int64_t)sz * c->ny + sy) * c->nx + sx];
                code = j >= 0 ? j : NB_SOLID;
            }
            nbr[(size_t)i * NW + (k - 1)] = code;
        }
    }
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

void apply_bc(lbms_ctx* c) {
    for (int s = 0; s < 3; ++s) c->L.xin[s] = c->x_in[s];
    outlet_flux_lattice(c->gas, c->current, c->L.q);
    if (c->periodic_x)
        for (int s = 0; s < 3; ++s) c->L.q[s] = 0.0;
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

// Copies a dense host field (3*N doubles) into X[cur] and restarts from the
// equilibrium f = w X (h = 0).
lbms_status upload_field(lbms_ctx* c, const double* X) {
    const int64_t S = c->L.S;
    const int nf = c->L.nf;
    std::vector<unsigned char> buf(3 * (size_t)S * x_size(c->L.precision), 0);
    for (int s = 0; s < 3; ++s)
        for (int i = 0; i < nf; ++i) put_x(c->L.precision, buf.data(), S, s * S + i, X[(size_t)s * c->N + c->fluid_cell[i]]);
    CK(cudaMemcpyAsync(c->L.b.X[c->L.cur], buf.data(), buf.size(), cudaMemcpyHostToDevice, c->stream),
       "upload mole fractions");
    c->h2d += buf.size();
    CK(launch_init(c->L, c->stream), "init kernel");
    CK(cudaStreamSynchronize(c->stream), "init");
    c->steps = 0;
    c->initialized = true;
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

lbms_status read_reduction(lbms_ctx* c, int slot, double* out, int nv) {
    CK(cudaMemcpyAsync(c->host_red, c->L.b.red_out + slot * kRedSlots, nv * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream),
       "reduction readback");
    CK(cudaStreamSynchronize(c->stream), "reduction");
    c->d2h += nv * sizeof(double);
    std::memcpy(out, c->host_red, nv * sizeof(double));
    return LBMS_OK;
}

}  // namespace

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

lbms_status lbms_create(const lbms_geometry* geom, const lbms_species* sp, const lbms_diffusivities* df, double T_K,
                        double p_Pa, const lbms_options* opt, lbms_ctx** out) {
    if (!out) return LBMS_EINVAL;
    *out = nullptr;
    t_create_error.clear();
    lbms_ctx* c = new (std::nothrow) lbms_ctx();
    if (!c) return LBMS_ENOMEM;
    lbms_status st = LBMS_OK;
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
    if (!geom) return bail(fail(c, LBMS_EINVAL, "geometry is NULL"));
    if (!sp) return bail(fail(c, LBMS_EINVAL, "species is NULL"));
    if (geom->dim != 2 && geom->dim != 3) return bail(fail(c, LBMS_EINVAL, "dim must be 2 or 3"));
    if (geom->nx < 1 || geom->ny < 1 || geom->nz < 1) return bail(fail(c, LBMS_EINVAL, "nx, ny, nz must be >= 1"));
    if (geom->dim == 2 && geom->nz != 1) return bail(fail(c, LBMS_EINVAL, "nz must be 1 when dim = 2"));
    if (!geom->periodic_x && geom->nx < 3) return bail(fail(c, LBMS_EINVAL, "nx must be >= 3 with an inlet and outlet"));
    if (!geom->solid) return bail(fail(c, LBMS_EINVAL, "solid mask is NULL"));
    if (!(geom->length_x_m > 0.0) || !std::isfinite(geom->length_x_m))
        return bail(fail(c, LBMS_EINVAL, "length_x_m must be finite and > 0"));
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

    c->dim = geom->dim;
    c->nx = geom->nx;
    c->ny = geom->ny;
    c->nz = geom->nz;
    c->Q = geom->dim == 2 ? D2Q9::Q : D3Q19::Q;
    c->periodic_x = geom->periodic_x ? 1 : 0;
    c->length_x = geom->length_x_m;
    c->N = (int64_t)c->nx * c->ny * c->nz;
    c->stream = static_cast<cudaStream_t>(c->opt.stream);

    // fluid cells, boundary columns
    std::vector<int> index_of((size_t)c->N, -1);
    for (int64_t cell = 0; cell < c->N; ++cell) {
        if (geom->solid[cell]) continue;
        if (c->fluid_cell.size() >= (size_t)std::numeric_limits<int>::max() / 2)
            return bail(fail(c, LBMS_EINVAL, "too many fluid cells for 32-bit indices"));
        index_of[cell] = (int)c->fluid_cell.size();
        c->fluid_cell.push_back(cell);
    }
    if (c->fluid_cell.empty()) return bail(fail(c, LBMS_EINVAL, "the mask has no fluid cell"));
    const int nrows = c->ny * c->nz;
    std::vector<int> rows(3 * (size_t)nrows, -1);
    for (int r = 0; r < nrows; ++r) {
        const int64_t base = (int64_t)r * c->nx;
        rows[r] = index_of[base];
        rows[nrows + r] = c->nx > 1 ? index_of[base + 1] : -1;
        rows[2 * nrows + r] = index_of[base + c->nx - 1];
        if (!c->periodic_x && (rows[r] < 0 || rows[2 * nrows + r] < 0))
            return bail(fail(c, LBMS_EINVAL, "inlet (x = 0) and outlet (x = nx-1) columns must be fluid"));
    }

    st = compute_props(c, sp, df, T_K, p_Pa);
    if (st != LBMS_OK) return bail(st);

    // device state
    Launch& L = c->L;
    L.dim = c->dim;
    L.precision = c->opt.precision;
    L.nf = (int)c->fluid_cell.size();
    L.S = ((int64_t)L.nf + 31) / 32 * 32;
    L.nrows = nrows;
    if ((int64_t)c->Q * L.S >= (int64_t)std::numeric_limits<int>::max())
        return bail(fail(c, LBMS_EINVAL, "too many fluid cells: Q x cells must stay below 2^31"));
    L.D12 = c->gas.D_lat[0][1];
    L.D13 = c->gas.D_lat[0][2];
    L.D23 = c->gas.D_lat[1][2];
    for (int s = 0; s < 3; ++s) L.stoich[s] = c->gas.stoich[s];
    L.tau_min = c->opt.tau_min;
    L.tau_max = c->opt.tau_max;
    L.drift = c->opt.coupling == LBMS_COUPLING_MS ? 1 : 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
    int smc = 0;
    if (cudaDeviceGetAttribute(&smc, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && smc > 0) L.sm_count = smc;
    e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "create capture stream"));
    e = cudaMallocHost(&c->host_red, 2 * kRedSlots * sizeof(double));
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "pinned readback buffer"));

    const size_t fbytes = (size_t)3 * c->Q * L.S * pop_size(L.precision);
    const size_t xbytes = (size_t)3 * L.S * x_size(L.precision);
    for (int k = 0; k < 2; ++k) {
        L.b.f[k] = dev_alloc(c, fbytes);
        L.b.X[k] = dev_alloc(c, xbytes);
    }
    const size_t sbytes = (size_t)3 * L.S * sizeof(double);
    L.b.snap = static_cast<double*>(dev_alloc(c, sbytes));
    const int nbw = c->dim == 2 ? nb_width<D2Q9>() : nb_width<D3Q19>();
    L.b.nbr = static_cast<int*>(dev_alloc(c, (size_t)nbw * L.S * sizeof(int)));
    L.b.rows = static_cast<int*>(dev_alloc(c, 3 * (size_t)nrows * sizeof(int)));
    L.b.red_partials = static_cast<double*>(dev_alloc(c, (size_t)kRedMaxBlocks * kRedSlots * sizeof(double)));
    L.b.red_counter = static_cast<unsigned int*>(dev_alloc(c, 4 * sizeof(unsigned int)));
    L.b.red_out = static_cast<double*>(dev_alloc(c, 2 * kRedSlots * sizeof(double)));
    if (!L.b.f[0] || !L.b.f[1] || !L.b.X[0] || !L.b.X[1] || !L.b.snap || !L.b.nbr || !L.b.rows ||
        !L.b.red_partials || !L.b.red_counter || !L.b.red_out)
        return bail(fail(c, LBMS_ENOMEM, "device allocation of %zu bytes failed", 2 * fbytes + 3 * xbytes));

    std::vector<int> nbr;
    if (c->dim == 2)
        build_neighbours<D2Q9>(c, index_of, L.S, nbr);
    else
        build_neighbours<D3Q19>(c, index_of, L.S, nbr);
    e = cudaMemcpyAsync(L.b.nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.b.rows, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.b.red_counter, 0, 4 * sizeof(unsigned int), c->stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(L.b.f[k], 0, fbytes, c->stream);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMemsetAsync(L.b.X[k], 0, xbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.b.snap, 0, sbytes, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "upload of the neighbour table"));
    c->h2d += nbr.size() * sizeof(int) + rows.size() * sizeof(int);
    *out = c;
    return LBMS_OK;
}

lbms_status lbms_set_bc(lbms_ctx* c, const double* x_inlet, double current_A_cm2) {
    if (!c || c->allocs.empty()) return fail(c, LBMS_ESTATE, "handle has no device state");
    lbms_status st = validate_bc(c, x_inlet, current_A_cm2);
    if (st != LBMS_OK) return st;
    for (int s = 0; s < 3; ++s) c->x_in[s] = x_inlet[s];
    c->current = current_A_cm2;
    apply_bc(c);
    drop_graphs(c);
    if (!c->initialized) {
        std::vector<double> X(3 * (size_t)c->N, 0.0);
        for (int s = 0; s < 3; ++s) std::fill(X.begin() + s * c->N, X.begin() + (s + 1) * c->N, c->x_in[s]);
        return upload_field(c, X.data());
    }
    return LBMS_OK;
}

lbms_status lbms_set_fields(lbms_ctx* c, const double* X) {
    if (!c || c->allocs.empty()) return fail(c, LBMS_ESTATE, "handle has no device state");
    if (!c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc before lbms_set_fields");
    if (!X) return fail(c, LBMS_EINVAL, "X is NULL");
    return upload_field(c, X);
}

lbms_status lbms_step(lbms_ctx* c, int64_t nsteps) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (nsteps < 0) return fail(c, LBMS_EINVAL, "nsteps must be >= 0");
    return launch_steps(c, nsteps);
}

lbms_status lbms_residual(lbms_ctx* c, int K, double* residual) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (K < 1 || !residual) return fail(c, LBMS_EINVAL, "need K >= 1 and a residual pointer");
    CK(launch_residual(c->L, 1, c->stream), "residual kernel");
    double r[10];
    lbms_status st = read_reduction(c, kRedResidual, r, 10);
    if (st != LBMS_OK) return st;
    if (r[9] > 0.0) {
        *residual = std::numeric_limits<double>::infinity();
        return fail(c, LBMS_EUNSTABLE, "%.0f non-finite mole fractions after %lld steps", r[9], (long long)c->steps);
    }
    double res = 0.0;
    for (int s = 0; s < 3; ++s)
        if (r[3 + s] > 0.0) res = std::max(res, std::sqrt(r[s]) / (K * std::sqrt(r[3 + s])));
    *residual = res;
    return LBMS_OK;
}

lbms_status lbms_run_to_residual(lbms_ctx* c, double tol, int64_t max_steps, int64_t* steps_taken,
                                 double* final_residual) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (!(tol >= 0.0) || max_steps < 0) return fail(c, LBMS_EINVAL, "need tol >= 0 and max_steps >= 0");
    const int K = c->opt.check_every;
    double r = std::numeric_limits<double>::infinity();
    int64_t done = 0;
    // the snapshot starts at the current state
    CK(launch_residual(c->L, 1, c->stream), "residual kernel");
    lbms_status st = LBMS_OK;
    while (done < max_steps) {
        const int64_t k = std::min<int64_t>(K, max_steps - done);
        st = launch_steps(c, k);
        if (st != LBMS_OK) break;
        done += k;
        st = lbms_residual(c, (int)k, &r);
        if (st != LBMS_OK) break;
        if (r <= tol) break;
    }
    if (steps_taken) *steps_taken = done;
    if (final_residual) *final_residual = r;
    if (st != LBMS_OK) return st;
    if (!(r <= tol)) return fail(c, LBMS_ENOTCONVERGED, "residual %.3e above %.3e after %lld steps", r, tol, (long long)done);
    return LBMS_OK;
}

lbms_status lbms_get_fields(lbms_ctx* c, double* X, double* u, double* tau) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    const int64_t S = c->L.S;
    const int nf = c->L.nf;
    const int prec = c->L.precision;
    if (X) {
        std::vector<unsigned char> b(3 * (size_t)S * x_size(prec));
        CK(cudaMemcpyAsync(b.data(), c->L.b.X[c->L.cur], b.size(), cudaMemcpyDeviceToHost, c->stream), "read X");
        CK(cudaStreamSynchronize(c->stream), "read X");
        c->d2h += b.size();
        std::fill(X, X + 3 * c->N, 0.0);
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i < nf; ++i) X[s * c->N + c->fluid_cell[i]] = get_x(prec, b.data(), S, s * S + i);
    }
    const size_t es = field_size(prec);
    auto to_double = [&](const std::vector<unsigned char>& b, int64_t idx) {
        return prec == LBMS_FP64 ? reinterpret_cast<const double*>(b.data())[idx]
                                 : (double)reinterpret_cast<const float*>(b.data())[idx];
    };
    if (u || tau) {
        if (!c->L.b.fields) {
            c->L.b.fields = dev_alloc(c, (size_t)(3 + 3 * c->dim) * S * es);
            if (!c->L.b.fields) return fail(c, LBMS_ENOMEM, "fields buffer");
        }
        CK(launch_fields(c->L, c->stream), "fields kernel");
        std::vector<unsigned char> b((size_t)(3 + 3 * c->dim) * S * es);
        CK(cudaMemcpyAsync(b.data(), c->L.b.fields, b.size(), cudaMemcpyDeviceToHost, c->stream), "read fields");
        CK(cudaStreamSynchronize(c->stream), "read fields");
        c->d2h += b.size();
        if (tau) {
            std::fill(tau, tau + 3 * c->N, 0.0);
            for (int s = 0; s < 3; ++s)
                for (int i = 0; i < nf; ++i) tau[s * c->N + c->fluid_cell[i]] = to_double(b, s * S + i);
        }
        if (u) {
            const double scale = c->gas.dx / c->gas.dt;
            std::fill(u, u + 3 * (size_t)c->dim * c->N, 0.0);
            for (int s = 0; s < 3; ++s)
                for (int d = 0; d < c->dim; ++d)
                    for (int i = 0; i < nf; ++i)
                        u[(s * c->dim + d) * c->N + c->fluid_cell[i]] =
                            scale * to_double(b, (3 + s * c->dim + d) * S + i);
        }
    }
    return LBMS_OK;
}

lbms_status lbms_overpotential(lbms_ctx* c, double* eta_V, double* x_out_mean) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (c->periodic_x) return fail(c, LBMS_EINVAL, "a box periodic in x has no outlet");
    CK(launch_boundary(c->L, c->stream), "boundary kernel");
    double r[6];
    lbms_status st = read_reduction(c, kRedBoundary, r, 6);
    if (st != LBMS_OK) return st;
    double xo[3];
    for (int s = 0; s < 3; ++s) xo[s] = r[3 + s] / c->L.nrows;
    if (x_out_mean)
        for (int s = 0; s < 3; ++s) x_out_mean[s] = xo[s];
    const double a = c->x_in[0] * xo[1];
    const double b = xo[0] * c->x_in[1];
    if (!(a > 0.0) || !(b > 0.0) || !std::isfinite(a) || !std::isfinite(b)) {
        if (eta_V) *eta_V = std::numeric_limits<double>::quiet_NaN();
        return fail(c, LBMS_EDEPLETED, "Eq. 43 undefined: X_in = (%g, %g), X_out = (%g, %g)", c->x_in[0], c->x_in[1],
                    xo[0], xo[1]);
    }
    if (eta_V) *eta_V = kR * c->gas.T / (c->gas.electrons * kF) * std::log(a / b);
    return LBMS_OK;
}

lbms_status lbms_boundary_flux(lbms_ctx* c, double* inlet_flux, double* totals) {
    if (!c || !c->initialized) return fail(c, LBMS_ESTATE, "call lbms_set_bc first");
    if (inlet_flux) {
        CK(launch_boundary(c->L, c->stream), "boundary kernel");
        double r[6];
        lbms_status st = read_reduction(c, kRedBoundary, r, 6);
        if (st != LBMS_OK) return st;
        for (int s = 0; s < 3; ++s) inlet_flux[s] = r[s];
    }
    if (totals) {
        CK(launch_residual(c->L, 0, c->stream), "sum kernel");
        double r[10];
        lbms_status st = read_reduction(c, kRedResidual, r, 10);
        if (st != LBMS_OK) return st;
        for (int s = 0; s < 3; ++s) totals[s] = r[6 + s];
    }
    return LBMS_OK;
}

lbms_status lbms_get_info(const lbms_ctx* c, lbms_info* info) {
    if (!c || !info) return LBMS_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->n_cells = c->N;
    info->n_fluid = (int64_t)c->fluid_cell.size();
    info->q = c->Q;
    info->precision = c->opt.precision;
    info->dx_m = c->gas.dx;
    info->dt_s = c->gas.dt;
    info->C_t = c->gas.C_t;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            info->D_eff_m2s[i * 3 + j] = c->gas.D_eff[i][j];
            info->D_lat[i * 3 + j] = c->gas.D_lat[i][j];
        }
    for (int s = 0; s < 3; ++s) {
        info->q_lat[s] = c->L.q[s];
        info->x_in[s] = c->x_in[s];
    }
    info->current_A_cm2 = c->current;
    info->steps = c->steps;
    info->device_bytes = c->device_bytes;
    info->h2d_bytes = c->h2d;
    info->d2h_bytes = c->d2h;
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
