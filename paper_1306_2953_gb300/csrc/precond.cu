// Preconditioners: none, the face-neighbour smoothing filter (the plain
// method's preconditioner; Sec. III cites a filter of Saad et al. without
// giving its form), and the learned convolutional network.
#include <new>

#include "device.h"
#include "ham.h"
#include "precond.h"

namespace rs {

int Precond::set_weights(const float *, const float *, const float *) {
    return fail(RS_EINVAL, "this preconditioner has no weights");
}

namespace {

class Identity : public Precond {
   public:
    int apply(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype,
              cudaStream_t st) override {
        return ham_filter(h, R, ldr, W, ldw, nb, dtype, 1.0, st);
    }
};

class Filter : public Precond {
   public:
    explicit Filter(double a) : alpha(a) {}
    int apply(const rs_ham *h, const void *R, int64_t ldr, void *W, int64_t ldw, int nb, int dtype,
              cudaStream_t st) override {
        return ham_filter(h, R, ldr, W, ldw, nb, dtype, alpha, st);
    }
    double alpha;
};

}  // namespace

Precond *Precond::create(int kind, double filter_alpha) {
    switch (kind) {
        case RS_PRECOND_NONE: return new (std::nothrow) Identity();
        case RS_PRECOND_FILTER: return new (std::nothrow) Filter(filter_alpha);
        default: return nullptr;
    }
}

}  // namespace rs
