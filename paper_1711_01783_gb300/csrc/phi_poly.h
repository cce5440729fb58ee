// Generated by gen_phi_poly.py -- polynomial pieces of phi(x) = -ln tanh(x/2).
// small branch x < 1.25: phi = ln2 - ln x - t*Ps(t), t = x^2
// large branch: phi = e*Pl(e^2), e = exp(-x)
#pragma once
#define MLD_PHI_X0 1.25f
// fit 'accurate': max |small fit error| 3.38e-09, max relative large fit error 4.63e-08
#define MLD_PHI_S0 (-8.333333104e-02f)
#define MLD_PHI_S1 (4.861036415e-03f)
#define MLD_PHI_S2 (-3.413196527e-04f)
#define MLD_PHI_S3 (2.552129118e-05f)
#define MLD_PHI_S4 (-1.561553869e-06f)
#define MLD_PHI_L0 (1.999999908e+00f)
#define MLD_PHI_L1 (6.667022306e-01f)
#define MLD_PHI_L2 (3.978680662e-01f)
#define MLD_PHI_L3 (3.259602744e-01f)
#define MLD_PHI2_Y0 1.8033688f
#define MLD_PHI2_C0 1.52876637f
// base-2 fit '2': max |small fit error| 1.59e-07 (bits), max relative large fit error 4.63e-08; max(small, large) relative error 1.46e-07 on [psi(lmax), lmax]
#define MLD_PHI2_S0 (-5.776221345e-02f)
#define MLD_PHI2_S1 (1.618349961e-03f)
#define MLD_PHI2_S2 (-5.385014368e-05f)
#define MLD_PHI2_S3 (1.586882831e-06f)
#define MLD_PHI2_L0 (2.885389949e+00f)
#define MLD_PHI2_L1 (9.618480019e-01f)
#define MLD_PHI2_L2 (5.740022860e-01f)
#define MLD_PHI2_L3 (4.702612714e-01f)
// base-2 fit '2H': max |small fit error| 1.93e-04 (bits), max relative large fit error 1.82e-04; max(small, large) relative error 2.03e-04 on [psi(lmax), lmax]
#define MLD_PHI2H_S0 (-5.769956003e-02f)
#define MLD_PHI2H_S1 (1.458956707e-03f)
#define MLD_PHI2H_L0 (2.884865946e+00f)
#define MLD_PHI2H_L1 (1.011935603e+00f)
