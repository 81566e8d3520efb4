// C ABI entry points (declared in include/nof.h): argument checks, workspace management and
// the orchestration of the device kernels for the set-up, the JK step, the energy+gradient
// evaluation and the optimiser step.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

static thread_local std::string g_last_error = "no error";

static std::atomic<long long> g_launches{0};

void nof_set_error(const std::string& msg) { g_last_error = msg; }
void nof_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

using EventPairs = std::vector<std::pair<cudaEvent_t, cudaEvent_t>>;

static void prof_clear(nof_ctx* c) {
    auto* ev = static_cast<EventPairs*>(c->prof_events);
    if (!ev) return;
    for (auto& e : *ev) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    ev->clear();
}

int prof_begin(nof_ctx* c, const char* name, int which) {
    if (c->prof_on != which) return NOF_OK;
    if (!c->prof_events) c->prof_events = new EventPairs();
    auto* ev = static_cast<EventPairs*>(c->prof_events);
    cudaEvent_t a, b;
    NOF_CUDA(cudaEventCreate(&a));
    NOF_CUDA(cudaEventCreate(&b));
    ev->push_back({a, b});
    c->prof_name = name;
    NOF_CUDA(cudaEventRecord(a, c->stream));
    return NOF_OK;
}

int prof_end(nof_ctx* c, int which) {
    if (c->prof_on != which) return NOF_OK;
    auto* ev = static_cast<EventPairs*>(c->prof_events);
    NOF_CUDA(cudaEventRecord(ev->back().second, c->stream));
    return NOF_OK;
}

int nof_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error '%s' (%d) in %s at %s:%d", cudaGetErrorString(e), (int)e,
             what, file, line);
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? NOF_ENOMEM : NOF_ECUDA;
}

namespace {

template <class T>
int dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        char buf[256];
        snprintf(buf, sizeof buf, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                 cudaGetErrorString(e));
        nof_set_error(buf);
        return NOF_ENOMEM;
    }
    return NOF_OK;
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

// Forget the recorded evaluation graphs (their kernels name workspaces that are about to change).
void drop_eval_graph(nof_ctx* c) {
    bool any = false;
    for (auto& g : c->geval) any = any || g.exec;
    if (any) cudaStreamSynchronize(c->stream);  // no replay still pending
    for (auto& g : c->geval) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = nof_ctx::EvalGraph{};
    }
    for (auto& k : c->gseen)
        for (auto& p : k) p = nullptr;
    c->gseen_next = 0;
}

void free_system(nof_ctx* c) {
    drop_eval_graph(c);
    if (c->fast) fast_release(c);
    dfree(c->fn_atom); dfree(c->fn_first); dfree(c->fn_nprim); dfree(c->pexp); dfree(c->pcoef);
    dfree(c->ax_atom); dfree(c->axexp); dfree(c->xyz); dfree(c->Z);
    dfree(c->S); dfree(c->H); dfree(c->vnn); dfree(c->B);
    dfree(c->pair); dfree(c->slot);
    dfree(c->T); dfree(c->b); dfree(c->d); dfree(c->J); dfree(c->K); dfree(c->D); dfree(c->W);
    dfree(c->HC); dfree(c->Lam); dfree(c->lam); dfree(c->hpp); dfree(c->A); dfree(c->Bc);
    dfree(c->s); dfree(c->t); dfree(c->ds); dfree(c->dt); dfree(c->occ); dfree(c->E);
    dfree(c->part); dfree(c->ggam); dfree(c->gorb);
    dfree(c->y); dfree(c->U); dfree(c->U2); dfree(c->tmpn); dfree(c->gwork);
    dfree(c->Dip); dfree(c->H0); dfree(c->vnn0); dfree(c->dipw); dfree(c->tdev);
    dfree(c->Linv); dfree(c->gr_cfit); dfree(c->gr_Y); dfree(c->gr_Gam); dfree(c->gr_Z); dfree(c->gr_small);
    dfree(c->opt_buf);
    c->opt_cap = 0;
    c->built = 0;
}

__global__ void k_unpack_sym(const double* Bp, int X, int n, double* B) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long nn = (long long)n * n;
    if (idx >= (long long)X * nn) return;
    long long P = idx / nn;
    long long r = idx - P * nn;
    int mu = (int)(r / n), nu = (int)(r % n);
    if (mu > nu) { int t = mu; mu = nu; nu = t; }
    long long npk = (long long)n * (n + 1) / 2;
    long long col = (long long)mu * n - (long long)mu * (mu - 1) / 2 + (nu - mu);
    B[idx] = Bp[P * npk + col];
}

bool basis_ok(const nof_basis* b) {
    if (!b || b->nshell <= 0 || !b->nprim || !b->exps) return false;
    int tot = 0;
    for (int s = 0; s < b->nshell; ++s) {
        if (b->nprim[s] <= 0) return false;
        tot += b->nprim[s];
    }
    for (int i = 0; i < tot; ++i)
        if (!(b->exps[i] > 0.0) || !std::isfinite(b->exps[i])) return false;
    return true;
}

int check_ctx(nof_ctx* c, bool need_built) {
    if (!c) {
        nof_set_error("null context");
        return NOF_EINVAL;
    }
    if (need_built && !c->built) {
        nof_set_error("nof_build_B has not been called on this context");
        return NOF_ESTATE;
    }
    return NOF_OK;
}

int run_jk(nof_ctx* c, const double* C) {
    if (c->opt.precision == NOF_PREC_SPLIT_BF16) return fast_jk(c, C);
    return plain_jk(c, C);
}
int run_grad(nof_ctx* c, const double* C, const double* gamma, bool want_grad) {
    if (c->opt.precision == NOF_PREC_SPLIT_BF16) return fast_grad(c, C, gamma, want_grad);
    return plain_grad(c, C, gamma, want_grad);
}

}  // namespace

extern "C" {

void nof_default_options(nof_options* o) {
    if (!o) return;
    o->ipnof = 7;
    o->isoftmax = 0;
    o->ncwo = 1;
    o->precision = NOF_PREC_FP64;
    o->on_iters = 20;
    o->on_lr = 0.3;
    o->lr = 0.02;
    o->b1 = 0.9;
    o->b2 = 0.999;
    o->eps = 1e-8;
    o->digits = 0;
    o->graphs = 1;
}

const char* nof_last_error(void) { return g_last_error.c_str(); }

int nof_create(nof_ctx** out, const nof_options* opt, void* stream) {
    if (!out) {
        nof_set_error("nof_create: null output pointer");
        return NOF_EINVAL;
    }
    *out = nullptr;
    nof_options o;
    nof_default_options(&o);
    if (opt) o = *opt;
    if (o.ipnof != 7 && o.ipnof != 5) {
        nof_set_error("nof_create: ipnof must be 5 or 7");
        return NOF_EINVAL;
    }
    if (o.isoftmax != 0 && o.isoftmax != 1) {
        nof_set_error("nof_create: isoftmax must be 0 (trigonometric mapping) or 1 (softmax mapping)");
        return NOF_EINVAL;
    }
    if (o.ncwo < 1 || o.on_iters < 0 ||
        (o.precision != NOF_PREC_FP64 && o.precision != NOF_PREC_SPLIT_BF16) ||
        (o.digits != 0 && o.digits != 4 && o.digits != 5) || (o.graphs != 0 && o.graphs != 1)) {
        nof_set_error("nof_create: bad ncwo, on_iters, precision, digits or graphs");
        return NOF_EINVAL;
    }
    nof_ctx* c = new (std::nothrow) nof_ctx;
    if (!c) {
        nof_set_error("nof_create: host allocation failed");
        return NOF_ENOMEM;
    }
    std::memset((void*)c, 0, sizeof(nof_ctx));
    c->opt = o;
    c->stream = (cudaStream_t)stream;
    int r = dalloc(&c->status, 1);
    if (r != NOF_OK) {
        delete c;
        return r;
    }
    cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
    cudaEvent_t* evs[8] = {&c->ev_fork, &c->ev_join, &c->ev_s0, &c->ev_sO, &c->ev_sT, &c->ev_sJ, &c->ev_s1, &c->ev_s2};
    for (cudaEvent_t* ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    int prio_low = 0, prio_high = 0;  // the side stream takes the lowest priority
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_low);
    if (e != cudaSuccess) {
        for (cudaEvent_t* ev : evs)
            if (*ev) cudaEventDestroy(*ev);
        if (c->side) cudaStreamDestroy(c->side);
        cudaFree(c->status);
        delete c;
        return nof_cuda_fail(e, "context set-up", __FILE__, __LINE__);
    }
    *out = c;
    return NOF_OK;
}

int nof_destroy(nof_ctx* c) {
    if (!c) return NOF_OK;
    cudaStreamSynchronize(c->stream);
    prof_clear(c);
    delete static_cast<EventPairs*>(c->prof_events);
    free_system(c);
    if (c->side) cudaStreamSynchronize(c->side);
    for (cudaEvent_t ev : {c->ev_fork, c->ev_join, c->ev_s0, c->ev_sO, c->ev_sT, c->ev_sJ, c->ev_s1, c->ev_s2})
        if (ev) cudaEventDestroy(ev);
    if (c->side) cudaStreamDestroy(c->side);
    dfree(c->status);
    delete c;
    return NOF_OK;
}

int nof_build_B(nof_ctx* c, int natom, const double* xyz, const double* Z, int charge, int mult,
                const nof_basis* orb, const nof_basis* aux) {
    NOF_TRY(check_ctx(c, false));
    if (natom <= 0 || !xyz || !basis_ok(orb) || !basis_ok(aux) || !orb->coefs) {
        nof_set_error("nof_build_B: bad geometry or basis");
        return NOF_EINVAL;
    }
    for (int i = 0; i < 3 * natom; ++i)
        if (!std::isfinite(xyz[i])) {
            nof_set_error("nof_build_B: non-finite coordinate");
            return NOF_ENONFINITE;
        }
    double ztot = 0.0;
    std::vector<double> hZ(natom, 1.0);
    if (Z)
        for (int i = 0; i < natom; ++i) hZ[i] = Z[i];
    for (double z : hZ) ztot += z;
    double ne = ztot - charge;
    int nelec = (int)std::lround(ne);
    if (mult != 1 || std::fabs(ne - nelec) > 1e-12 || nelec <= 0 || nelec % 2) {
        nof_set_error("nof_build_B: only closed-shell singlets (mult = 1, even electron count)");
        return NOF_EINVAL;
    }
    // host description of the basis, functions ordered atom by atom
    std::vector<int> fn_atom, fn_first, fn_nprim, ax_atom;
    std::vector<double> pexp, pcoef, axexp;
    for (int A = 0; A < natom; ++A) {
        int off = 0;
        for (int s = 0; s < orb->nshell; ++s) {
            fn_atom.push_back(A);
            fn_first.push_back((int)pexp.size());
            fn_nprim.push_back(orb->nprim[s]);
            for (int k = 0; k < orb->nprim[s]; ++k) {
                pexp.push_back(orb->exps[off + k]);
                pcoef.push_back(orb->coefs[off + k]);
            }
            off += orb->nprim[s];
        }
        off = 0;
        for (int s = 0; s < aux->nshell; ++s) {
            for (int k = 0; k < aux->nprim[s]; ++k) {
                ax_atom.push_back(A);
                axexp.push_back(aux->exps[off + k]);
            }
            off += aux->nprim[s];
        }
    }
    const int n = (int)fn_atom.size(), X = (int)ax_atom.size();
    const int npair = nelec / 2, ncwo = c->opt.ncwo;
    const int a = npair * (ncwo + 1);
    if (a > n) {
        nof_set_error("nof_build_B: N/2 (ncwo + 1) exceeds the number of basis functions");
        return NOF_EINVAL;
    }
    std::vector<int> pair(a, -1), slot(a, -1);
    for (int g = 0; g < npair; ++g) {
        pair[g] = g;
        slot[g] = 0;
        for (int i = 1; i <= ncwo; ++i) {
            int p = npair + (i - 1) * npair + (npair - 1 - g);
            pair[p] = g;
            slot[p] = i;
        }
    }
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    free_system(c);
    c->natom = natom; c->nbf = n; c->naux = X; c->nact = a; c->npair = npair;
    c->nelec = nelec; c->ngamma = npair * ncwo;
    const size_t nn = (size_t)n * n, aa = (size_t)a * a, na = (size_t)n * a;
    const size_t npk = (size_t)n * (n + 1) / 2;
    // system description
    NOF_TRY(dalloc(&c->fn_atom, n)); NOF_TRY(dalloc(&c->fn_first, n)); NOF_TRY(dalloc(&c->fn_nprim, n));
    NOF_TRY(dalloc(&c->pexp, pexp.size())); NOF_TRY(dalloc(&c->pcoef, pcoef.size()));
    NOF_TRY(dalloc(&c->ax_atom, X)); NOF_TRY(dalloc(&c->axexp, X));
    NOF_TRY(dalloc(&c->xyz, 3 * (size_t)natom)); NOF_TRY(dalloc(&c->Z, natom));
    NOF_TRY(dalloc(&c->pair, a)); NOF_TRY(dalloc(&c->slot, a));
    cudaStream_t st = c->stream;
    NOF_CUDA(cudaMemcpyAsync(c->fn_atom, fn_atom.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->fn_first, fn_first.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->fn_nprim, fn_nprim.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->pexp, pexp.data(), pexp.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->pcoef, pcoef.data(), pcoef.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->ax_atom, ax_atom.data(), X * sizeof(int), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->axexp, axexp.data(), X * sizeof(double), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->xyz, xyz, 3 * (size_t)natom * sizeof(double), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->Z, hZ.data(), natom * sizeof(double), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->pair, pair.data(), a * sizeof(int), cudaMemcpyHostToDevice, st));
    NOF_CUDA(cudaMemcpyAsync(c->slot, slot.data(), a * sizeof(int), cudaMemcpyHostToDevice, st));
    // one-electron data and the RI tensor
    NOF_TRY(dalloc(&c->S, nn)); NOF_TRY(dalloc(&c->H, nn)); NOF_TRY(dalloc(&c->vnn, 1));
    NOF_TRY(dalloc(&c->B, (size_t)X * nn));
    double *M3 = nullptr, *V2 = nullptr, *Linv = nullptr, *Bp = nullptr;
    int r = dalloc(&M3, (size_t)X * npk);
    if (r == NOF_OK) r = dalloc(&V2, (size_t)X * X);
    if (r == NOF_OK) r = dalloc(&Linv, (size_t)X * X);
    if (r == NOF_OK) r = dalloc(&Bp, (size_t)X * npk);
    if (r == NOF_OK) r = build_integrals(c, M3, V2);
    if (r == NOF_OK) {
        cudaError_t e = cudaMemsetAsync(c->status, 0, sizeof(int), st);
        if (e != cudaSuccess) r = nof_cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
    }
    if (r == NOF_OK) r = cholesky_inverse(V2, Linv, X, c->status, st);
    int hstat = 0;
    if (r == NOF_OK) {
        cudaError_t e = cudaMemcpyAsync(&hstat, c->status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = nof_cuda_fail(e, "status readback", __FILE__, __LINE__);
        else if (hstat & NOF_DEV_ILLCOND) {
            nof_set_error("nof_build_B: the auxiliary Coulomb metric is numerically singular");
            r = NOF_EILLCOND;
            cudaMemsetAsync(c->status, 0, sizeof(int), st);
        }
    }
    if (r == NOF_OK) {  // Bp = L^{-1} M3 over the packed pair index
        Gemm64 g;
        g.M = X; g.N = (int)npk; g.K = X;
        g.A = Linv; g.sAm = X; g.sAk0 = 1; g.a_lower = true;
        g.B = M3; g.sBn = 1; g.sBk0 = (long long)npk;
        g.C = Bp; g.sCm = (long long)npk; g.sCn = 1;
        r = gemm64(g, st);
    }
    if (r == NOF_OK) {
        long long tot = (long long)X * nn;
        k_unpack_sym<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Bp, X, n, c->B);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) r = nof_cuda_fail(e, "k_unpack_sym", __FILE__, __LINE__);
    }
    if (r == NOF_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) r = nof_cuda_fail(e, "build sync", __FILE__, __LINE__);
    }
    cudaFree(M3); cudaFree(V2); cudaFree(Bp);
    if (r == NOF_OK && c->opt.precision == NOF_PREC_FP64)
        c->Linv = Linv;  // kept for the nuclear gradient's fitting coefficients
    else
        cudaFree(Linv);
    if (r != NOF_OK) {
        free_system(c);
        return r;
    }
    // evaluation workspaces
    int splits_cap = 304;
    c->part_elems = (size_t)splits_cap * na;
    const bool plain = c->opt.precision == NOF_PREC_FP64;
    NOF_TRY(dalloc(&c->T, plain ? (size_t)X * na : 1));
    NOF_TRY(dalloc(&c->b, plain ? (size_t)X * aa : 1));
    NOF_TRY(dalloc(&c->W, plain ? (size_t)X * aa + c->part_elems : 1));
    NOF_TRY(dalloc(&c->d, (size_t)X * a)); NOF_TRY(dalloc(&c->D, (size_t)X * a));
    NOF_TRY(dalloc(&c->J, aa)); NOF_TRY(dalloc(&c->K, aa)); NOF_TRY(dalloc(&c->A, aa)); NOF_TRY(dalloc(&c->Bc, aa));
    NOF_TRY(dalloc(&c->HC, na)); NOF_TRY(dalloc(&c->Lam, na));
    NOF_TRY(dalloc(&c->lam, nn)); NOF_TRY(dalloc(&c->gorb, nn));
    NOF_TRY(dalloc(&c->hpp, a)); NOF_TRY(dalloc(&c->s, a)); NOF_TRY(dalloc(&c->t, a)); NOF_TRY(dalloc(&c->occ, a));
    NOF_TRY(dalloc(&c->ds, (size_t)a * ncwo)); NOF_TRY(dalloc(&c->dt, (size_t)a * ncwo));
    NOF_TRY(dalloc(&c->E, 1)); NOF_TRY(dalloc(&c->part, 4 * (size_t)a)); NOF_TRY(dalloc(&c->ggam, c->ngamma));
    NOF_TRY(dalloc(&c->y, nn)); NOF_TRY(dalloc(&c->U, nn)); NOF_TRY(dalloc(&c->U2, nn)); NOF_TRY(dalloc(&c->tmpn, nn));
    NOF_TRY(dalloc(&c->tdev, 1));  // device-side step counter (nof_step with t == NULL)
    NOF_CUDA(cudaMemsetAsync(c->tdev, 0, sizeof(int), c->stream));
    {   // split-K scratch for the small FP64 GEMMs (n x n, n x a, a x a, X x a outputs)
        size_t big = nn > (size_t)X * a ? nn : (size_t)X * a;
        size_t cap = 304 * big;
        if (cap > ((size_t)32 << 20)) cap = (size_t)32 << 20;
        c->gwork_cap = cap;
        NOF_TRY(dalloc(&c->gwork, cap));
    }
    if (!plain) {
        r = fast_prepare(c);
        if (r != NOF_OK) {
            free_system(c);
            return r;
        }
        dfree(c->B);  // the split path keeps only the digit planes of B
    }
    c->built = 1;
    return NOF_OK;
}

int nof_query(nof_ctx* c, int* nbf, int* naux, int* nact, int* ngamma, double* vnn) {
    NOF_TRY(check_ctx(c, true));
    if (nbf) *nbf = c->nbf;
    if (naux) *naux = c->naux;
    if (nact) *nact = c->nact;
    if (ngamma) *ngamma = c->ngamma;
    if (vnn) {
        NOF_CUDA(cudaMemcpyAsync(vnn, c->vnn, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        NOF_CUDA(cudaStreamSynchronize(c->stream));
    }
    return NOF_OK;
}

int nof_get_SH(nof_ctx* c, double* S, double* H) {
    NOF_TRY(check_ctx(c, true));
    size_t bytes = (size_t)c->nbf * c->nbf * sizeof(double);
    if (S) NOF_CUDA(cudaMemcpyAsync(S, c->S, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (H) NOF_CUDA(cudaMemcpyAsync(H, c->H, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return NOF_OK;
}

int nof_split_digits(nof_ctx* c, int* nd) {
    NOF_TRY(check_ctx(c, true));
    if (!nd || !c->fast) {
        nof_set_error("nof_split_digits: null output or not a split-precision context");
        return NOF_EINVAL;
    }
    *nd = fast_digits(c);
    return NOF_OK;
}

int nof_tuned_tiles(nof_ctx* c, int* out) {
    NOF_TRY(check_ctx(c, true));
    if (!out || !c->fast) {
        nof_set_error("nof_tuned_tiles: null output or not a split-precision context");
        return NOF_EINVAL;
    }
    return fast_tiles(c, out);
}

int nof_get_B(nof_ctx* c, double* B) {
    NOF_TRY(check_ctx(c, true));
    if (!B) {
        nof_set_error("nof_get_B: null output");
        return NOF_EINVAL;
    }
    if (c->opt.precision == NOF_PREC_SPLIT_BF16) return fast_get_B(c, B);
    size_t bytes = (size_t)c->naux * c->nbf * c->nbf * sizeof(double);
    NOF_CUDA(cudaMemcpyAsync(B, c->B, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return NOF_OK;
}

int nof_lowdin(nof_ctx* c, const double* Q, double* C) {
    NOF_TRY(check_ctx(c, true));
    if (!Q || !C) {
        nof_set_error("nof_lowdin: null pointer");
        return NOF_EINVAL;
    }
    const int n = c->nbf;
    // workspaces: y, U, U2, tmpn as Newton-Schulz scratch, lam as the result S^{-1/2}
    NOF_TRY(newton_schulz_invsqrt(c->S, c->lam, c->y, c->U, c->U2, c->tmpn, n, 40, c->stream, c->gwork,
                                  c->gwork_cap));
    Gemm64 g;
    g.M = n; g.N = n; g.K = n;
    g.A = c->lam; g.sAm = n; g.sAk0 = 1;
    g.B = Q; g.sBn = 1; g.sBk0 = n;
    g.C = C; g.sCm = n; g.sCn = 1;
    return gemm64(g, c->stream);
}

int nof_core_guess(nof_ctx* c, double* C0, double* eps) {
    NOF_TRY(check_ctx(c, true));
    if (!C0) {
        nof_set_error("nof_core_guess: null output");
        return NOF_EINVAL;
    }
    const int n = c->nbf;
    cudaStream_t st = c->stream;
    // X = S^{-1/2} into lam; A = X^T H X into U (via tmpn = H X); eigenvectors into y; C0 = X y
    NOF_TRY(newton_schulz_invsqrt(c->S, c->lam, c->y, c->U, c->U2, c->tmpn, n, 40, st, c->gwork, c->gwork_cap));
    Gemm64 g;
    g.M = n; g.N = n; g.K = n;
    g.A = c->H; g.sAm = n; g.sAk0 = 1;
    g.B = c->lam; g.sBn = 1; g.sBk0 = n;
    g.C = c->tmpn; g.sCm = n; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    NOF_TRY(gemm64(g, st));
    g.A = c->lam; g.sAm = 1; g.sAk0 = n;  // X^T (X is symmetric; written generally)
    g.B = c->tmpn; g.sBn = 1; g.sBk0 = n;
    g.C = c->U;
    NOF_TRY(gemm64(g, st));
    double* w = eps ? eps : c->gorb;  // eigenvalues (scratch when the caller does not want them)
    NOF_TRY(sym_eig(c->U, c->U2, c->y, w, n, (int*)c->part, st));
    g.A = c->lam; g.sAm = n; g.sAk0 = 1;
    g.B = c->y; g.sBn = 1; g.sBk0 = n;
    g.C = C0;
    return gemm64(g, st);
}

int nof_jk(nof_ctx* c, const double* C, double* J, double* K) {
    NOF_TRY(check_ctx(c, true));
    if (!C || !J || !K) {
        nof_set_error("nof_jk: null pointer");
        return NOF_EINVAL;
    }
    NOF_TRY(run_jk(c, C));
    size_t bytes = (size_t)c->nact * c->nact * sizeof(double);
    NOF_CUDA(cudaMemcpyAsync(J, c->J, bytes, cudaMemcpyDeviceToDevice, c->stream));
    NOF_CUDA(cudaMemcpyAsync(K, c->K, bytes, cudaMemcpyDeviceToDevice, c->stream));
    return NOF_OK;
}

// One evaluation, every kernel launched on the context's stream.
static int energy_grad_body(nof_ctx* c, const double* C, const double* gamma, double* E, double* g_orb,
                            double* g_gamma) {
    const bool grad = g_orb || g_gamma;
    if (c->opt.precision == NOF_PREC_SPLIT_BF16) {
        NOF_TRY(fast_eval(c, C, gamma, grad));
    } else {
        NOF_TRY(run_jk(c, C));
        NOF_TRY(run_grad(c, C, gamma, grad));
    }
    if (E) NOF_CUDA(cudaMemcpyAsync(E, c->E, sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (g_orb)
        NOF_CUDA(cudaMemcpyAsync(g_orb, c->gorb, (size_t)c->nbf * c->nbf * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->stream));
    if (g_gamma)
        NOF_CUDA(cudaMemcpyAsync(g_gamma, c->ggam, (size_t)c->ngamma * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->stream));
    return NOF_OK;
}

int nof_energy_grad(nof_ctx* c, const double* C, const double* gamma, double* E, double* g_orb,
                    double* g_gamma) {
    NOF_TRY(check_ctx(c, true));
    if (!C || !gamma) {
        nof_set_error("nof_energy_grad: null C or gamma");
        return NOF_EINVAL;
    }
    if (!c->opt.graphs || !c->stream || c->prof_on || c->gfail)
        return energy_grad_body(c, C, gamma, E, g_orb, g_gamma);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NOF_CUDA(cudaStreamIsCapturing(c->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) return energy_grad_body(c, C, gamma, E, g_orb, g_gamma);
    const void* key[5] = {C, gamma, E, g_orb, g_gamma};
    auto same_as = [&](const void* const* k) {
        for (int i = 0; i < 5; ++i)
            if (k[i] != key[i]) return false;
        return true;
    };
    nof_ctx::EvalGraph* hit = nullptr;
    for (auto& g : c->geval)
        if (g.exec && same_as(g.key)) hit = &g;
    if (!hit) {
        int seen = -1;
        for (int s = 0; s < nof_ctx::kEvalGraphs; ++s)
            if (same_as(c->gseen[s])) seen = s;
        if (seen < 0) {  // new pointers: run directly and remember them (the graphs stay)
            for (int i = 0; i < 5; ++i) c->gseen[c->gseen_next][i] = key[i];
            c->gseen_next = (c->gseen_next + 1) % nof_ctx::kEvalGraphs;
            return energy_grad_body(c, C, gamma, E, g_orb, g_gamma);
        }
        // second call with these pointers: record the evaluation into the least recently used
        // slot, then replay it below
        for (int i = 0; i < 5; ++i) c->gseen[seen][i] = nullptr;
        hit = nullptr;  // an empty slot, else the least recently used one
        for (auto& g : c->geval)
            if (!hit && !g.exec) hit = &g;
        if (!hit) {
            hit = &c->geval[0];
            for (auto& g : c->geval)
                if (g.used < hit->used) hit = &g;
        }
        if (hit->exec) {
            cudaStreamSynchronize(c->stream);  // no replay of the replaced graph still pending
            cudaGraphExecDestroy(hit->exec);
            *hit = nof_ctx::EvalGraph{};
        }
        const long long l0 = g_launches.load();
        NOF_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int r = energy_grad_body(c, C, gamma, E, g_orb, g_gamma);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        const long long recorded = g_launches.load() - l0;
        g_launches.fetch_sub(recorded);  // counted again at each replay
        if (r == NOF_OK && e == cudaSuccess) e = cudaGraphInstantiate(&hit->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (r != NOF_OK || e != cudaSuccess) {
            // recording failed: nothing ran, so run directly and keep launching directly from now on
            hit->exec = nullptr;
            c->gfail = 1;
            cudaGetLastError();
            return energy_grad_body(c, C, gamma, E, g_orb, g_gamma);
        }
        for (int i = 0; i < 5; ++i) hit->key[i] = key[i];
        hit->kernels = recorded;
    }
    hit->used = ++c->gtick;
    NOF_CUDA(cudaGraphLaunch(hit->exec, c->stream));
    g_launches.fetch_add(hit->kernels);
    return NOF_OK;
}

int nof_step(nof_ctx* c, double* C, double* gamma, double* m, double* v, int* t, double* out) {
    NOF_TRY(check_ctx(c, true));
    if (!C || !gamma || !m || !v || !out) {
        nof_set_error("nof_step: null pointer");
        return NOF_EINVAL;
    }
    NOF_TRY(run_jk(c, C));
    NOF_TRY(pnof_on_update(c, gamma));
    NOF_TRY(run_grad(c, C, gamma, true));
    return pnof_adam_rotate(c, C, m, v, t, out);
}

int nof_energy_grad_batch(nof_ctx* const* ctxs, int count, const double* const* C, const double* const* gamma,
                          double* const* E, double* const* g_orb, double* const* g_gamma, void* stream) {
    if (count <= 0 || !ctxs || !C || !gamma || !E) {
        nof_set_error("nof_energy_grad_batch: bad count or null array");
        return NOF_EINVAL;
    }
    for (int i = 0; i < count; ++i) {
        NOF_TRY(check_ctx(ctxs[i], true));
        if (!C[i] || !gamma[i] || !E[i]) {
            nof_set_error("nof_energy_grad_batch: null C, gamma or E entry");
            return NOF_EINVAL;
        }
    }
    cudaStream_t master = (cudaStream_t)stream;
    NOF_CUDA(cudaEventRecord(ctxs[0]->ev_fork, master));
    for (int i = 0; i < count; ++i) {
        nof_ctx* c = ctxs[i];
        NOF_CUDA(cudaStreamWaitEvent(c->stream, ctxs[0]->ev_fork, 0));
        NOF_TRY(nof_energy_grad(c, C[i], gamma[i], E[i], g_orb ? g_orb[i] : nullptr,
                                g_gamma ? g_gamma[i] : nullptr));
        NOF_CUDA(cudaEventRecord(c->ev_join, c->stream));
        NOF_CUDA(cudaStreamWaitEvent(master, c->ev_join, 0));
    }
    return NOF_OK;
}

long long nof_kernel_launches(void) { return g_launches.load(); }

int nof_profile(nof_ctx* c, int enable) {
    NOF_TRY(check_ctx(c, false));
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    if (enable < 0 || enable > 3) {
        nof_set_error("nof_profile: enable must be 0 (off) or 1..3 (the contraction to time)");
        return NOF_EINVAL;
    }
    prof_clear(c);
    c->prof_name = nullptr;
    c->prof_on = enable;
    return NOF_OK;
}

int nof_profile_read(nof_ctx* c, double* ms, int* launches, const char** name) {
    NOF_TRY(check_ctx(c, false));
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    int cnt = 0;
    if (auto* ev = static_cast<EventPairs*>(c->prof_events)) {
        for (auto& e : *ev) {
            float t = 0.f;
            NOF_CUDA(cudaEventElapsedTime(&t, e.first, e.second));
            tot += t;
            ++cnt;
        }
    }
    if (ms) *ms = tot;
    if (launches) *launches = cnt;
    if (name) *name = c->prof_name ? c->prof_name : "";
    return NOF_OK;
}

int nof_sync(nof_ctx* c) {
    NOF_TRY(check_ctx(c, false));
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    int h = 0;
    NOF_CUDA(cudaMemcpy(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        NOF_CUDA(cudaMemset(c->status, 0, sizeof(int)));
        if (h & NOF_DEV_TIMEOUT) {
            nof_set_error("a bounded device-side wait timed out");
            return NOF_ETIMEOUT;
        }
        if (h & NOF_DEV_NONFINITE) {
            nof_set_error("non-finite value detected on the device");
            return NOF_ENONFINITE;
        }
        if (h & NOF_DEV_ILLCOND) {
            nof_set_error("ill-conditioned metric");
            return NOF_EILLCOND;
        }
        if (h & NOF_DEV_RANGE) {
            nof_set_error("a step's rotation exceeded the fixed scaling of the device-counter step "
                          "(||y||_F > 4096)");
            return NOF_ENOTCONV;
        }
    }
    return NOF_OK;
}

}  // extern "C"
