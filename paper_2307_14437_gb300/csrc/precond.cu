// Sparse preconditioner of Section 3.3 (placeholder until the IC factor lands).
#include "gofd_internal.cuh"

namespace gofd {

struct Precond {
    int pattern = 0;
    double shift = 0;
    int64_t nnz = 0;
};

void setup_precond(gofd_problem* p) {
    if (p->opt.precond == 0) return;
    fail(GOFD_E_ARG, "preconditioner not available in this build");
}

void free_precond(gofd_problem* p) {
    delete p->pc;
    p->pc = nullptr;
}

int64_t precond_nnz(const gofd_problem* p) { return p->pc ? p->pc->nnz : 0; }
double precond_shift(const gofd_problem* p) { return p->pc ? p->pc->shift : 0.0; }

void precond_apply(gofd_problem*, bool, const void*, void*, cudaStream_t) {
    fail(GOFD_E_ARG, "no preconditioner");
}

}  // namespace gofd
