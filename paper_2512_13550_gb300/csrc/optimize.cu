// nof_optimize: the converged ON / NO optimisation loop on one context.
//
// The paper optimises the ONs and the NOs separately (Theory section, after Eq. sum1): the ONs
// fully at fixed orbitals, the orbitals by rotations C <- C exp(y) with ADAM on the orbital
// gradient g = 4(lambda - lambda^T) (Natural Orbital Optimization subsection), until the
// lambda-symmetry and energy thresholds are met (NTHRESHL / NTHRESHE, Single Point Energy
// section). The ADAM details are delegated to another publication; the loop here is the reading
// the oracle implements (oracle/optimize.py):
//   outer iteration k: J, K, h_pp at C_k; ONs converged at fixed J, K by BFGS (k_on_bfgs); E_k and
//   g_k at (C_k, gamma_k); stop when ||g_k|| < gtol and |E_k - E_{k-1}| < etol; else `maxloop` ADAM
//   steps from zero moments with gamma_k fixed, each a full evaluation, keeping the best orbitals
//   (lower energy by more than etol, or equal within etol with ||g|| at most 0.9 of the best); the rate halves
//   when no step is better than the start; the loop also ends once the rate is below lr_min.
// Every step of the loop runs in the library's kernels on the context's stream; the host reads
// back three numbers per evaluation (E, ||g||, max |lambda - lambda^T|) to take the decisions.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace {

int eval_jk(nof_ctx* c, const double* C) {
    return c->opt.precision == NOF_PREC_SPLIT_BF16 ? fast_jk(c, C) : plain_jk(c, C);
}
int eval_grad(nof_ctx* c, const double* C, const double* gamma) {
    return c->opt.precision == NOF_PREC_SPLIT_BF16 ? fast_grad(c, C, gamma, true) : plain_grad(c, C, gamma, true);
}

// C_out = C_in exp(y) (U scratch in c->U; the exponential and the product on the context's stream)
int rotate(nof_ctx* c, const double* Cin, const double* y, double* Cout) {
    const int n = c->nbf;
    NOF_TRY(expm_antisym_device(y, c->U, c->U2, c->tmpn, n, c->stream, c->gwork, c->gwork_cap));
    Gemm64 g;
    g.M = n; g.N = n; g.K = n;
    g.A = Cin; g.sAm = n; g.sAk0 = 1;
    g.B = c->U; g.sBn = 1; g.sBk0 = n;
    g.C = Cout; g.sCm = n; g.sCn = 1;
    g.work = c->gwork; g.work_cap = c->gwork_cap;
    return gemm64(g, c->stream);
}

// ---- L-BFGS on the rotation generators (the refinement phase) -----------------------------------
// Inner product of antisymmetric matrices <A, B> = sum_{p<q} A_pq B_pq = (1/2) sum A o B. A dot
// product is kDotBlocks block partials written by k_dot_part; its consumers add them in a fixed
// order (dot64), so every value is deterministic and no host synchronisation is needed.
constexpr int kDotBlocks = 64;

__global__ void __launch_bounds__(256) k_dot_part(const double* a, const double* b, long long nn, double* part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < nn; i += (long long)kDotBlocks * 256) acc += a[i] * b[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void __launch_bounds__(256) k_absmax_part(const double* a, long long nn, double* part) {
    __shared__ double red[256];
    double m = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < nn; i += (long long)kDotBlocks * 256) m = fmax(m, fabs(a[i]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__device__ __forceinline__ double dot64(const double* part) {
    double s = 0.0;
    for (int i = 0; i < kDotBlocks; ++i) s += part[i];
    return 0.5 * s;
}
__device__ __forceinline__ double max64(const double* part) {
    double m = 0.0;
    for (int i = 0; i < kDotBlocks; ++i) m = fmax(m, part[i]);
    return m;
}
// first loop of the two-loop recursion: a_i = rho_i <s_i, q> (stored), q -= a_i y_i
__global__ void k_lbfgs_down(double* q, const double* y, const double* part, const double* rho, double* a_out,
                             long long nn) {
    const double a = *rho * dot64(part);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i == 0) *a_out = a;
    if (i < nn) q[i] -= a * y[i];
}
// second loop: b = rho_i <y_i, q>, q += (a_i - b) s_i
__global__ void k_lbfgs_up(double* q, const double* s, const double* part, const double* rho, const double* a_i,
                           long long nn) {
    const double b = *rho * dot64(part);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) q[i] += (*a_i - b) * s[i];
}
// q *= <s, y> / <y, y> of the newest pair (the initial inverse-Hessian scale), from its stored dots
__global__ void k_lbfgs_scale(double* q, const double* sy, const double* yy, long long nn) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) q[i] *= *sy / *yy;
}
// d = -q, or the steepest-descent start d = -g lr / max|g| (max from k_absmax_part partials)
__global__ void k_negate(double* d, const double* q, long long nn) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) d[i] = -q[i];
}
__global__ void k_steepest(double* d, const double* g, const double* part_max, double lr, long long nn) {
    const double s = lr / max64(part_max);
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) d[i] = -g[i] * s;
}
// out = alpha x; diff = a - b
__global__ void k_scaled(double* out, const double* x, double alpha, long long nn) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) out[i] = alpha * x[i];
}
__global__ void k_diff(double* out, const double* a, const double* b, long long nn) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) out[i] = a[i] - b[i];
}
// a new pair: sy = <s, y>, yy = <y, y>, rho = 1 / sy into slot scalars (the host tests sy > 0 first)
__global__ void k_pair_scalars(const double* part_sy, const double* part_yy, double* sy, double* yy, double* rho) {
    const double a = dot64(part_sy), b = dot64(part_yy);
    *sy = a;
    *yy = b;
    *rho = 1.0 / a;
}

inline unsigned blocks(long long n) { return (unsigned)((n + 255) / 256); }

// A non-finite energy or gradient ends the loop with NOF_ENONFINITE: the status bit the energy
// kernel set is cleared, since the return value reports it.
int non_finite(nof_ctx* c, const char* msg) {
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    NOF_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    nof_set_error(msg);
    return NOF_ENONFINITE;
}

int read_host(nof_ctx* c, double* dst, const double* src, int count) {
    NOF_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
    NOF_CUDA(cudaStreamSynchronize(c->stream));
    return NOF_OK;
}

}  // namespace

extern "C" {

void nof_default_opt_params(nof_opt_params* p) {
    if (!p) return;
    p->maxit = 1000;
    p->maxloop = 10;
    p->gtol = 1e-5;
    p->etol = 1e-8;
    p->lr = 0.02;
    p->lr_min = 1e-12;
    p->on_tol = 1e-8;
    p->on_maxit = 500;
    p->eps_rel = 0.0;
    p->lr_grow = 1.0;
    p->orbopt = 2;
    p->memory = 20;
    p->lbfgs_after = 1.0 / 64.0;
}

int nof_optimize(nof_ctx* c, double* C, double* gamma, const nof_opt_params* prm, double* history, double* result) {
    if (!c || !C || !gamma || !result) {
        nof_set_error("nof_optimize: null context, C, gamma or result");
        return NOF_EINVAL;
    }
    if (!c->built) {
        nof_set_error("nof_build_B has not been called on this context");
        return NOF_ESTATE;
    }
    nof_opt_params p;
    nof_default_opt_params(&p);
    if (prm) p = *prm;
    if (p.maxit < 1 || p.maxloop < 1 || !(p.gtol > 0.0) || !(p.etol >= 0.0) || !(p.lr > 0.0) ||
        !(p.lr_min >= 0.0) || !(p.on_tol > 0.0) || p.on_maxit < 0 || !(p.eps_rel >= 0.0) || !(p.lr_grow >= 1.0) ||
        p.orbopt < 0 || p.orbopt > 2 || p.memory < 1 || p.memory > 64 || !(p.lbfgs_after >= 0.0)) {
        nof_set_error("nof_optimize: bad parameters (maxit, maxloop >= 1; gtol, lr, on_tol > 0; orbopt 0..2; "
                      "memory 1..64)");
        return NOF_EINVAL;
    }
    const int n = c->nbf, ng = c->ngamma;
    const size_t nn = (size_t)n * n;
    const int mem = p.orbopt ? p.memory : 0;
    // [Ccur | Cbest | m | v | g | y] n^2 each, [E | stats 3 | info 2], BFGS scratch 6 ng + ng^2,
    // L-BFGS pairs 2 mem n^2, scalars (dot partials, per-pair <s,y>, <y,y>, rho, a)
    const size_t nscal = (size_t)kDotBlocks * 4 + 4 * 64;
    const size_t need = 6 * nn + 8 + 6 * (size_t)ng + (size_t)ng * ng + 2 * (size_t)mem * nn + nscal;
    if (c->opt_cap < need) {
        if (c->opt_buf) cudaFree(c->opt_buf);
        c->opt_buf = nullptr;
        c->opt_cap = 0;
        NOF_CUDA(cudaMalloc((void**)&c->opt_buf, need * sizeof(double)));
        c->opt_cap = need;
    }
    double* Ccur = c->opt_buf;
    double* Cbest = Ccur + nn;
    double* m = Cbest + nn;
    double* v = m + nn;
    double* gbuf = v + nn;
    double* y = gbuf + nn;
    double* Ed = y + nn;
    double* stats = Ed + 1;
    double* info = stats + 3;
    double* w = info + 2;
    double* Smem = w + 6 * (size_t)ng + (size_t)ng * ng;  // L-BFGS s_i, y_i: slot j at Smem + j nn
    double* Ymem = Smem + (size_t)mem * nn;
    double* part = Ymem + (size_t)mem * nn;  // 4 dot-partial buffers of kDotBlocks
    double* part2 = part + kDotBlocks;
    double* part3 = part2 + kDotBlocks;
    double* part4 = part3 + kDotBlocks;
    double* psy = part4 + kDotBlocks;  // per slot <s, y>, <y, y>, rho, a
    double* pyy = psy + 64;
    double* prho = pyy + 64;
    double* pa = prho + 64;
    cudaStream_t st = c->stream;
    const unsigned nb = blocks((long long)nn);
    // L-BFGS state: the pairs live in slots of a ring, oldest first from `first`
    int npairs = 0, first = 0;
    bool use_lbfgs = p.orbopt == 1;
    double* gk = m;  // during L-BFGS steps the ADAM buffers hold g_k and the direction d
    double* dir = v;
    auto dot_host = [&](const double* a, const double* b, double* out) -> int {
        k_dot_part<<<kDotBlocks, 256, 0, st>>>(a, b, (long long)nn, part4);
        NOF_LAUNCH_CHECK();
        double h64[kDotBlocks];
        NOF_CUDA(cudaMemcpyAsync(h64, part4, sizeof h64, cudaMemcpyDeviceToHost, st));
        NOF_CUDA(cudaStreamSynchronize(st));
        double sum = 0.0;
        for (int i = 0; i < kDotBlocks; ++i) sum += h64[i];  // dot64's order
        *out = 0.5 * sum;
        return NOF_OK;
    };
    // d = -H g by the two-loop recursion over the stored pairs, or -g lr / max|g| without pairs
    auto direction = [&](double lr_now) -> int {
        if (npairs == 0) {
            k_absmax_part<<<kDotBlocks, 256, 0, st>>>(gk, (long long)nn, part);
            NOF_LAUNCH_CHECK();
            k_steepest<<<nb, 256, 0, st>>>(dir, gk, part, lr_now, (long long)nn);
            NOF_LAUNCH_CHECK();
            return NOF_OK;
        }
        double* q = y;  // scratch
        NOF_CUDA(cudaMemcpyAsync(q, gk, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
        for (int j = npairs - 1; j >= 0; --j) {
            const int slot = (first + j) % mem;
            k_dot_part<<<kDotBlocks, 256, 0, st>>>(Smem + slot * nn, q, (long long)nn, part);
            NOF_LAUNCH_CHECK();
            k_lbfgs_down<<<nb, 256, 0, st>>>(q, Ymem + slot * nn, part, prho + slot, pa + slot, (long long)nn);
            NOF_LAUNCH_CHECK();
        }
        const int newest = (first + npairs - 1) % mem;
        k_lbfgs_scale<<<nb, 256, 0, st>>>(q, psy + newest, pyy + newest, (long long)nn);
        NOF_LAUNCH_CHECK();
        for (int j = 0; j < npairs; ++j) {
            const int slot = (first + j) % mem;
            k_dot_part<<<kDotBlocks, 256, 0, st>>>(Ymem + slot * nn, q, (long long)nn, part);
            NOF_LAUNCH_CHECK();
            k_lbfgs_up<<<nb, 256, 0, st>>>(q, Smem + slot * nn, part, prho + slot, pa + slot, (long long)nn);
            NOF_LAUNCH_CHECK();
        }
        k_negate<<<nb, 256, 0, st>>>(dir, q, (long long)nn);
        NOF_LAUNCH_CHECK();
        return NOF_OK;
    };

    double lr = p.lr, E_prev = 0.0, h[3] = {0.0, 0.0, 0.0}, hinfo[2] = {0.0, 0.0};
    long long evals = 0, on_steps = 0;
    int k = 0, converged = 0;
    for (k = 0; k < p.maxit; ++k) {
        // ONs converged at C_k, then E_k and g_k
        NOF_TRY(eval_jk(c, C));
        NOF_TRY(pnof_on_converge(c, gamma, p.on_tol, p.on_maxit, c->opt.on_lr, w, info));
        NOF_TRY(eval_grad(c, C, gamma));
        NOF_TRY(pnof_step_stats(c, c->gorb, stats));
        NOF_TRY(read_host(c, h, stats, 3));
        NOF_TRY(read_host(c, hinfo, info, 2));
        ++evals;
        on_steps += (long long)hinfo[0];
        if (!std::isfinite(h[0]) || !std::isfinite(h[1])) {
            result[0] = h[0];
            result[1] = h[1];
            return non_finite(c, "nof_optimize: non-finite energy or gradient");
        }
        if (history) {
            history[3 * k] = h[0];
            history[3 * k + 1] = h[1];
            history[3 * k + 2] = lr;
        }
        if (h[1] < p.gtol && k > 0 && std::fabs(h[0] - E_prev) < p.etol) {
            converged = 1;
            ++k;
            break;
        }
        if (lr < p.lr_min) {
            ++k;
            break;
        }
        E_prev = h[0];
        if (p.orbopt == 2 && !use_lbfgs && lr < p.lr * p.lbfgs_after) use_lbfgs = true;
        if (use_lbfgs) {
            // one L-BFGS step at gamma_k fixed: the direction from the stored pairs, the step length
            // by halving from 1: Armijo where the predicted decrease exceeds etol, else a smaller
            // ||g|| with the energy within etol; then, once, the same from steepest descent
            NOF_CUDA(cudaMemcpyAsync(gk, c->gorb, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
            NOF_TRY(direction(lr));
            double dg = 0.0;
            NOF_TRY(dot_host(dir, gk, &dg));
            if (dg >= 0.0) {
                npairs = 0;
                NOF_TRY(direction(lr));
                NOF_TRY(dot_host(dir, gk, &dg));
            }
            bool accepted = false;
            double alpha = 1.0;
            for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
                alpha = 1.0;
                for (int ls = 0; ls < 12; ++ls) {
                    k_scaled<<<nb, 256, 0, st>>>(y, dir, alpha, (long long)nn);
                    NOF_LAUNCH_CHECK();
                    NOF_TRY(rotate(c, C, y, c->tmpn));
                    NOF_CUDA(cudaMemcpyAsync(Ccur, c->tmpn, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
                    NOF_TRY(nof_energy_grad(c, Ccur, gamma, Ed, gbuf, nullptr));
                    NOF_TRY(pnof_step_stats(c, gbuf, stats));
                    double e[3];
                    NOF_TRY(read_host(c, e, stats, 3));
                    ++evals;
                    if (!std::isfinite(e[0]) || !std::isfinite(e[1]))
                        return non_finite(c, "nof_optimize: non-finite energy or gradient in an orbital step");
                    const bool ok = (-alpha * dg > p.etol) ? (e[0] <= h[0] + 1e-4 * alpha * dg)
                                                           : (e[0] <= h[0] + p.etol && e[1] < h[1]);
                    if (ok) {
                        accepted = true;
                        break;
                    }
                    alpha *= 0.5;
                }
                if (accepted || npairs == 0) break;
                npairs = 0;
                NOF_TRY(direction(lr));
                NOF_TRY(dot_host(dir, gk, &dg));
            }
            if (!accepted) {
                lr *= 0.5;
                continue;
            }
            NOF_CUDA(cudaMemcpyAsync(C, Ccur, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
            // the pair s = alpha d (still in y from the accepted trial), y = g(trial) - g_k (into
            // Cbest, unused by these steps), kept when <s, y> > 0 in the next ring slot (the oldest
            // one once the ring is full)
            k_diff<<<nb, 256, 0, st>>>(Cbest, gbuf, gk, (long long)nn);
            NOF_LAUNCH_CHECK();
            double sy = 0.0;
            NOF_TRY(dot_host(y, Cbest, &sy));
            if (sy > 0.0) {
                const int slot = npairs < mem ? (first + npairs) % mem : first;
                double* sv = Smem + (size_t)slot * nn;
                double* yv = Ymem + (size_t)slot * nn;
                NOF_CUDA(cudaMemcpyAsync(sv, y, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
                NOF_CUDA(cudaMemcpyAsync(yv, Cbest, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
                k_dot_part<<<kDotBlocks, 256, 0, st>>>(sv, yv, (long long)nn, part2);
                NOF_LAUNCH_CHECK();
                k_dot_part<<<kDotBlocks, 256, 0, st>>>(yv, yv, (long long)nn, part3);
                NOF_LAUNCH_CHECK();
                k_pair_scalars<<<1, 1, 0, st>>>(part2, part3, psy + slot, pyy + slot, prho + slot);
                NOF_LAUNCH_CHECK();
                if (npairs < mem) ++npairs;
                else first = (first + 1) % mem;
            }
            continue;
        }
        // a block of ADAM steps from zero moments with gamma_k fixed, keeping the lowest-energy
        // orbitals
        NOF_CUDA(cudaMemsetAsync(m, 0, 2 * nn * sizeof(double), st));  // m and v
        NOF_CUDA(cudaMemcpyAsync(gbuf, c->gorb, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
        NOF_CUDA(cudaMemcpyAsync(Ccur, C, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
        // a step is better than the best so far when its energy is lower by more than etol, or
        // equal within etol with a ||g|| at most 0.9 of the best (energies that close are compared
        // through the gradient, which the split-precision path resolves far better than the energy)
        double best_e = h[0], best_g = h[1];
        bool improved = false;
        const double eps = std::max(c->opt.eps, p.eps_rel * h[1]);  // relative to ||g_k|| if eps_rel > 0
        for (int t = 1; t <= p.maxloop; ++t) {
            NOF_TRY(pnof_adam_y(c, gbuf, m, v, y, t, lr, eps));
            NOF_TRY(rotate(c, Ccur, y, c->tmpn));  // C exp(y) into tmpn, then back into Ccur
            NOF_CUDA(cudaMemcpyAsync(Ccur, c->tmpn, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
            NOF_TRY(nof_energy_grad(c, Ccur, gamma, Ed, gbuf, nullptr));
            NOF_TRY(pnof_step_stats(c, gbuf, stats));
            double e[3];
            NOF_TRY(read_host(c, e, stats, 3));
            ++evals;
            if (!std::isfinite(e[0]) || !std::isfinite(e[1]))
                return non_finite(c, "nof_optimize: non-finite energy or gradient in an orbital step");
            if (e[0] < best_e - p.etol || (std::fabs(e[0] - best_e) <= p.etol && e[1] < 0.9 * best_g)) {
                best_e = e[0];
                best_g = e[1];
                improved = true;
                NOF_CUDA(cudaMemcpyAsync(Cbest, Ccur, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
            }
        }
        if (improved) {
            NOF_CUDA(cudaMemcpyAsync(C, Cbest, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
            lr *= p.lr_grow;
        } else {
            lr *= 0.5;
        }
    }
    NOF_CUDA(cudaStreamSynchronize(st));
    result[0] = h[0];
    result[1] = h[1];
    result[2] = h[2];
    result[3] = (double)k;
    result[4] = (double)evals;
    result[5] = (double)converged;
    result[6] = lr;
    result[7] = (double)on_steps;
    return NOF_OK;
}

}  // extern "C"
