// Solver entry points that are not built yet report PC_ESTATE.
#include <cmath>

#include "pc_internal.h"

using namespace pc;

namespace pc {
void release_solver_state(pc_grid*) {}
int precond_set_k(pc_grid*) { return PC_OK; }
}  // namespace pc

extern "C" {

int pc_options_default(pc_options* o) {
    if (!o) return fail(PC_EINVAL, "pc_options_default: null");
    o->tol = 1e-8;
    o->inner_tol = 1e-10;
    o->precision = PC_PREC_FP64;
    o->full_space = 0;
    o->block_size = 4;
    o->max_basis = 32;
    o->max_restarts = 60;
    o->inner_maxit = 400;
    o->guard = 3;
    o->verbose = 0;
    return PC_OK;
}

double pc_default_sigma(const pc_grid* g) {
    if (!g) return NAN;
    double cmax = 0, rmax = 0;
    for (int p = 0; p < 2; ++p) {
        for (int e = 0; e < 36; ++e) cmax = std::fmax(cmax, std::fabs(g->Chat[p][e]));
        rmax = std::fmax(rmax, g->rhohat[p]);
    }
    return -0.30 * cmax / rmax;
}

int pc_block_fourier(pc_grid*, int, int, int, const void*, void*, void*) {
    return fail(PC_ESTATE, "pc_block_fourier: not available in this build");
}

int pc_shift_invert_pcg(pc_grid*, int, int, double, const void*, void*, double, int, pc_pcg_info*, void*) {
    return fail(PC_ESTATE, "pc_shift_invert_pcg: not available in this build");
}

int pc_eigs(pc_grid*, const double*, int, double, const pc_options*, double*, void*, int*, pc_eigs_info*) {
    return fail(PC_ESTATE, "pc_eigs: not available in this build");
}

}  // extern "C"
