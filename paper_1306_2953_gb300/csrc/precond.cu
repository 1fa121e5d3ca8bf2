// Preconditioners: none, the face-neighbour smoothing filter (the plain
// method's preconditioner; Sec. III cites a filter of Saad et al. without
// giving its form), the learned convolutional network, and a few conjugate-
// gradient iterations on the shifted Poisson operator that the network is
// trained to imitate.
#include <new>

#include "device.h"
#include "ham.h"
#include "learned.h"
#include "precond.h"

namespace rs {

int Precond::set_weights(const float *, cudaStream_t) {
    return fail(RS_EINVAL, "this preconditioner has no weights");
}

namespace {

class Identity : public Precond {
   public:
    int apply(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype,
              cudaStream_t st) override {
        return ham_filter(h, R, ldr, W, ldw, nb, dtype, 1.0, st);
    }
    int kind() const override { return RS_PRECOND_NONE; }
};

class Filter : public Precond {
   public:
    explicit Filter(double a) : alpha(a) {}
    int apply(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype,
              cudaStream_t st) override {
        return ham_filter(h, R, ldr, W, ldw, nb, dtype, alpha, st);
    }
    int kind() const override { return RS_PRECOND_FILTER; }
    double alpha;
};

// The learned network (learned.cu); FP32 residuals only.
class Learned : public Precond {
   public:
    int init(int64_t npts, int nb) {
        RS_TRY(w.alloc(sizeof(float) * LEARNED_WEIGHTS));
        RS_TRY(wq.alloc(sizeof(float) * LEARNED_WEIGHTS));
        RS_TRY(dots.alloc(sizeof(double) * 128));
        return act.alloc(sizeof(float) * (size_t)learned_act_floats(npts, nb));
    }
    int set_weights(const float *w_dev, cudaStream_t st) override {
        RS_CUDA(cudaMemcpyAsync(w.p, w_dev, sizeof(float) * LEARNED_WEIGHTS, cudaMemcpyDeviceToDevice, st));
        RS_TRY(learned_round_weights(w.as<float>(), wq.as<float>(), st));
        ready = true;
        return RS_OK;
    }
    int apply(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype,
              cudaStream_t st) override {
        if (!ready) return fail(RS_EINVAL, "learned preconditioner: weights not set");
        if (dtype != RS_F32) return fail(RS_EINVAL, "learned preconditioner: FP32 residuals only");
        return learned_apply(h, (const float *)R, ldr, (float *)W, ldw, nb, wq.as<float>(), act.as<float>(),
                             dots.as<double>(), st);
    }
    int kind() const override { return RS_PRECOND_LEARNED; }
    DevBuf w, wq, act, dots;
    bool ready = false;
};

// A few CG iterations on (-1/2 Lap + sigma) W = R, into a scratch block
// [npts][nb] and then into W (whose leading dimension may differ).
class ShiftedCG : public Precond {
   public:
    int init(rs_ham *hs, int iters, int64_t n, int b, int dtype) {
        shifted = hs;
        n_iter = iters;
        npts = n;
        nb = b;
        es = dtype == RS_F64 ? 8 : 4;
        RS_TRY(x.alloc((size_t)npts * nb * es));
        return work.alloc((size_t)rs_cg_workspace_bytes(npts, nb, dtype));
    }
    int apply(const rs_ham *, const void *R, int64_t ldr, void *W, int64_t ldw, int ncols, int dtype,
              cudaStream_t st) override {
        if (ldr != nb || ncols != nb) return fail(RS_EINVAL, "CG preconditioner: residual block must be [npts][nb]");
        RS_TRY(rs_shifted_poisson_cg(shifted, R, x.p, nb, nb, n_iter, dtype, work.p, st));
        RS_CUDA(cudaMemcpy2DAsync(W, (size_t)ldw * es, x.p, (size_t)nb * es, (size_t)nb * es, (size_t)npts,
                                  cudaMemcpyDeviceToDevice, st));
        return RS_OK;
    }
    int kind() const override { return RS_PRECOND_CG; }
    rs_ham *shifted = nullptr;
    int n_iter = 0, nb = 1, es = 4;
    int64_t npts = 0;
    DevBuf x, work;
};

}  // namespace

Precond *Precond::create_cg(rs_ham *shifted, int n_iter, int64_t npts, int nb, int dtype) {
    ShiftedCG *p = new (std::nothrow) ShiftedCG();
    if (!p) return nullptr;
    if (p->init(shifted, n_iter, npts, nb, dtype) != RS_OK) {
        delete p;
        return nullptr;
    }
    return p;
}

Precond *Precond::create(int kind, double filter_alpha, int64_t npts, int nb, int dtype) {
    switch (kind) {
        case RS_PRECOND_NONE: return new (std::nothrow) Identity();
        case RS_PRECOND_FILTER: return new (std::nothrow) Filter(filter_alpha);
        case RS_PRECOND_LEARNED: {
            if (dtype != RS_F32) return nullptr;
            Learned *l = new (std::nothrow) Learned();
            if (l && l->init(npts, nb) != RS_OK) {
                delete l;
                return nullptr;
            }
            return l;
        }
        default: return nullptr;
    }
}

}  // namespace rs
