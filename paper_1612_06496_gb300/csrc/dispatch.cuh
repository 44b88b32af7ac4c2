// Run-time embedding dimension -> compile-time template argument.
// The row kernels keep a row's d values in registers, so d is a template
// parameter; these are the dimensions built into the library.
#pragma once

#define PFE_D_CASE(DV, ...)       \
    case DV: {                    \
        constexpr int D = DV;     \
        __VA_ARGS__;              \
    } break;

#define PFE_DISPATCH_D(dval, ...)                                                     \
    switch (dval) {                                                                   \
        PFE_D_CASE(1, __VA_ARGS__) PFE_D_CASE(2, __VA_ARGS__) PFE_D_CASE(3, __VA_ARGS__) \
        PFE_D_CASE(4, __VA_ARGS__) PFE_D_CASE(5, __VA_ARGS__) PFE_D_CASE(6, __VA_ARGS__) \
        PFE_D_CASE(7, __VA_ARGS__) PFE_D_CASE(8, __VA_ARGS__) PFE_D_CASE(9, __VA_ARGS__) \
        PFE_D_CASE(10, __VA_ARGS__) PFE_D_CASE(11, __VA_ARGS__) PFE_D_CASE(12, __VA_ARGS__) \
        PFE_D_CASE(13, __VA_ARGS__) PFE_D_CASE(14, __VA_ARGS__) PFE_D_CASE(15, __VA_ARGS__) \
        PFE_D_CASE(16, __VA_ARGS__) PFE_D_CASE(20, __VA_ARGS__) PFE_D_CASE(24, __VA_ARGS__) \
        PFE_D_CASE(25, __VA_ARGS__) PFE_D_CASE(32, __VA_ARGS__)                          \
        default:                                                                      \
            return PFE_EUNSUPPORTED;                                                  \
    }                                                                                 \
    return PFE_EUNSUPPORTED;
