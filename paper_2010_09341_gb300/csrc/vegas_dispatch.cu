// vegas_dispatch.cu -- sampling-kernel lookup by (mode, family, d, layout).
#include "vegas_kernels.cuh"

namespace vegas {

const void *sample_kernel_f64_const(int d, bool priv);
const void *sample_kernel_f64_sum(int d, bool priv);
const void *sample_kernel_f64_gauss_sym(int d, bool priv);
const void *sample_kernel_f64_genz_osc(int d, bool priv);
const void *sample_kernel_f64_genz_gauss(int d, bool priv);
const void *sample_kernel_f64_genz_prod(int d, bool priv);
const void *sample_kernel_f64_genz_corner(int d, bool priv);
const void *sample_kernel_f64_lo(int d, bool priv);
const void *sample_kernel_f64_lo_pdf(int d, bool priv);
const void *sample_kernel_f32sum64_const(int d, bool priv);
const void *sample_kernel_f32sum64_sum(int d, bool priv);
const void *sample_kernel_f32sum64_gauss_sym(int d, bool priv);
const void *sample_kernel_f32sum64_genz_osc(int d, bool priv);
const void *sample_kernel_f32sum64_genz_gauss(int d, bool priv);
const void *sample_kernel_f32sum64_genz_prod(int d, bool priv);
const void *sample_kernel_f32sum64_genz_corner(int d, bool priv);
const void *sample_kernel_f32sum64_lo(int d, bool priv);
const void *sample_kernel_f32sum64_lo_pdf(int d, bool priv);
const void *sample_kernel_f32kahan_const(int d, bool priv);
const void *sample_kernel_f32kahan_sum(int d, bool priv);
const void *sample_kernel_f32kahan_gauss_sym(int d, bool priv);
const void *sample_kernel_f32kahan_genz_osc(int d, bool priv);
const void *sample_kernel_f32kahan_genz_gauss(int d, bool priv);
const void *sample_kernel_f32kahan_genz_prod(int d, bool priv);
const void *sample_kernel_f32kahan_genz_corner(int d, bool priv);
const void *sample_kernel_f32kahan_lo(int d, bool priv);
const void *sample_kernel_f32kahan_lo_pdf(int d, bool priv);

const void *sample_strat_kernel_f64_const(int d, bool priv);
const void *sample_strat_kernel_f64_sum(int d, bool priv);
const void *sample_strat_kernel_f64_gauss_sym(int d, bool priv);
const void *sample_strat_kernel_f64_genz_osc(int d, bool priv);
const void *sample_strat_kernel_f64_genz_gauss(int d, bool priv);
const void *sample_strat_kernel_f64_genz_prod(int d, bool priv);
const void *sample_strat_kernel_f64_genz_corner(int d, bool priv);
const void *sample_strat_kernel_f64_lo(int d, bool priv);
const void *sample_strat_kernel_f64_lo_pdf(int d, bool priv);
const void *sample_strat_kernel_f32sum64_const(int d, bool priv);
const void *sample_strat_kernel_f32sum64_sum(int d, bool priv);
const void *sample_strat_kernel_f32sum64_gauss_sym(int d, bool priv);
const void *sample_strat_kernel_f32sum64_genz_osc(int d, bool priv);
const void *sample_strat_kernel_f32sum64_genz_gauss(int d, bool priv);
const void *sample_strat_kernel_f32sum64_genz_prod(int d, bool priv);
const void *sample_strat_kernel_f32sum64_genz_corner(int d, bool priv);
const void *sample_strat_kernel_f32sum64_lo(int d, bool priv);
const void *sample_strat_kernel_f32sum64_lo_pdf(int d, bool priv);
const void *sample_strat_kernel_f32kahan_const(int d, bool priv);
const void *sample_strat_kernel_f32kahan_sum(int d, bool priv);
const void *sample_strat_kernel_f32kahan_gauss_sym(int d, bool priv);
const void *sample_strat_kernel_f32kahan_genz_osc(int d, bool priv);
const void *sample_strat_kernel_f32kahan_genz_gauss(int d, bool priv);
const void *sample_strat_kernel_f32kahan_genz_prod(int d, bool priv);
const void *sample_strat_kernel_f32kahan_genz_corner(int d, bool priv);
const void *sample_strat_kernel_f32kahan_lo(int d, bool priv);
const void *sample_strat_kernel_f32kahan_lo_pdf(int d, bool priv);

const void *sample_kernel_f64_const_wide(int d);
const void *sample_kernel_f64_sum_wide(int d);
const void *sample_kernel_f64_gauss_sym_wide(int d);
const void *sample_kernel_f64_genz_osc_wide(int d);
const void *sample_kernel_f64_genz_gauss_wide(int d);
const void *sample_kernel_f64_genz_prod_wide(int d);
const void *sample_kernel_f64_genz_corner_wide(int d);
const void *sample_kernel_f64_lo_wide(int d);

// The FP64 kernels with one histogram copy per lane (pick_family_wide), or
// null where there is none (another mode, the density-grid family, d > 16).
const void *sample_kernel_wide(int mode, int fam, int d) {
    if (mode != ACC_F64) return nullptr;
    switch (fam) {
    case F_CONST: return sample_kernel_f64_const_wide(d);
    case F_SUM: return sample_kernel_f64_sum_wide(d);
    case F_GAUSS_SYM: return sample_kernel_f64_gauss_sym_wide(d);
    case F_GENZ_OSC: return sample_kernel_f64_genz_osc_wide(d);
    case F_GENZ_GAUSS: return sample_kernel_f64_genz_gauss_wide(d);
    case F_GENZ_PROD: return sample_kernel_f64_genz_prod_wide(d);
    case F_GENZ_CORNER: return sample_kernel_f64_genz_corner_wide(d);
    case F_LO: return sample_kernel_f64_lo_wide(d);
    default: return nullptr;
    }
}

const void *sample_kernel(int mode, int fam, int d, bool priv) {
    switch (mode) {
    case ACC_F64:
        switch (fam) {
        case F_CONST: return sample_kernel_f64_const(d, priv);
        case F_SUM: return sample_kernel_f64_sum(d, priv);
        case F_GAUSS_SYM: return sample_kernel_f64_gauss_sym(d, priv);
        case F_GENZ_OSC: return sample_kernel_f64_genz_osc(d, priv);
        case F_GENZ_GAUSS: return sample_kernel_f64_genz_gauss(d, priv);
        case F_GENZ_PROD: return sample_kernel_f64_genz_prod(d, priv);
        case F_GENZ_CORNER: return sample_kernel_f64_genz_corner(d, priv);
        case F_LO: return sample_kernel_f64_lo(d, priv);
        case F_LO_PDF: return sample_kernel_f64_lo_pdf(d, priv);
        default: return nullptr;
        }
    case ACC_F32_SUM64:
        switch (fam) {
        case F_CONST: return sample_kernel_f32sum64_const(d, priv);
        case F_SUM: return sample_kernel_f32sum64_sum(d, priv);
        case F_GAUSS_SYM: return sample_kernel_f32sum64_gauss_sym(d, priv);
        case F_GENZ_OSC: return sample_kernel_f32sum64_genz_osc(d, priv);
        case F_GENZ_GAUSS: return sample_kernel_f32sum64_genz_gauss(d, priv);
        case F_GENZ_PROD: return sample_kernel_f32sum64_genz_prod(d, priv);
        case F_GENZ_CORNER: return sample_kernel_f32sum64_genz_corner(d, priv);
        case F_LO: return sample_kernel_f32sum64_lo(d, priv);
        case F_LO_PDF: return sample_kernel_f32sum64_lo_pdf(d, priv);
        default: return nullptr;
        }
    case ACC_F32_KAHAN:
        switch (fam) {
        case F_CONST: return sample_kernel_f32kahan_const(d, priv);
        case F_SUM: return sample_kernel_f32kahan_sum(d, priv);
        case F_GAUSS_SYM: return sample_kernel_f32kahan_gauss_sym(d, priv);
        case F_GENZ_OSC: return sample_kernel_f32kahan_genz_osc(d, priv);
        case F_GENZ_GAUSS: return sample_kernel_f32kahan_genz_gauss(d, priv);
        case F_GENZ_PROD: return sample_kernel_f32kahan_genz_prod(d, priv);
        case F_GENZ_CORNER: return sample_kernel_f32kahan_genz_corner(d, priv);
        case F_LO: return sample_kernel_f32kahan_lo(d, priv);
        case F_LO_PDF: return sample_kernel_f32kahan_lo_pdf(d, priv);
        default: return nullptr;
        }
    default: return nullptr;
    }
}

const void *sample_strat_kernel(int mode, int fam, int d, bool priv) {
    switch (mode) {
    case ACC_F64:
        switch (fam) {
        case F_CONST: return sample_strat_kernel_f64_const(d, priv);
        case F_SUM: return sample_strat_kernel_f64_sum(d, priv);
        case F_GAUSS_SYM: return sample_strat_kernel_f64_gauss_sym(d, priv);
        case F_GENZ_OSC: return sample_strat_kernel_f64_genz_osc(d, priv);
        case F_GENZ_GAUSS: return sample_strat_kernel_f64_genz_gauss(d, priv);
        case F_GENZ_PROD: return sample_strat_kernel_f64_genz_prod(d, priv);
        case F_GENZ_CORNER: return sample_strat_kernel_f64_genz_corner(d, priv);
        case F_LO: return sample_strat_kernel_f64_lo(d, priv);
        case F_LO_PDF: return sample_strat_kernel_f64_lo_pdf(d, priv);
        default: return nullptr;
        }
    case ACC_F32_SUM64:
        switch (fam) {
        case F_CONST: return sample_strat_kernel_f32sum64_const(d, priv);
        case F_SUM: return sample_strat_kernel_f32sum64_sum(d, priv);
        case F_GAUSS_SYM: return sample_strat_kernel_f32sum64_gauss_sym(d, priv);
        case F_GENZ_OSC: return sample_strat_kernel_f32sum64_genz_osc(d, priv);
        case F_GENZ_GAUSS: return sample_strat_kernel_f32sum64_genz_gauss(d, priv);
        case F_GENZ_PROD: return sample_strat_kernel_f32sum64_genz_prod(d, priv);
        case F_GENZ_CORNER: return sample_strat_kernel_f32sum64_genz_corner(d, priv);
        case F_LO: return sample_strat_kernel_f32sum64_lo(d, priv);
        case F_LO_PDF: return sample_strat_kernel_f32sum64_lo_pdf(d, priv);
        default: return nullptr;
        }
    case ACC_F32_KAHAN:
        switch (fam) {
        case F_CONST: return sample_strat_kernel_f32kahan_const(d, priv);
        case F_SUM: return sample_strat_kernel_f32kahan_sum(d, priv);
        case F_GAUSS_SYM: return sample_strat_kernel_f32kahan_gauss_sym(d, priv);
        case F_GENZ_OSC: return sample_strat_kernel_f32kahan_genz_osc(d, priv);
        case F_GENZ_GAUSS: return sample_strat_kernel_f32kahan_genz_gauss(d, priv);
        case F_GENZ_PROD: return sample_strat_kernel_f32kahan_genz_prod(d, priv);
        case F_GENZ_CORNER: return sample_strat_kernel_f32kahan_genz_corner(d, priv);
        case F_LO: return sample_strat_kernel_f32kahan_lo(d, priv);
        case F_LO_PDF: return sample_strat_kernel_f32kahan_lo_pdf(d, priv);
        default: return nullptr;
        }
    default: return nullptr;
    }
}

}  // namespace vegas
