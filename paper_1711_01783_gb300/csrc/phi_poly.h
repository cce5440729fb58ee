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
// base-2 fit '2': max |small fit error| 5.05e-09 (bits), max relative large fit error 4.63e-08
#define MLD_PHI2_S0 (-5.776226393e-02f)
#define MLD_PHI2_S1 (1.618846898e-03f)
#define MLD_PHI2_S2 (-5.461420978e-05f)
#define MLD_PHI2_S3 (1.962797304e-06f)
#define MLD_PHI2_S4 (-5.779495718e-08f)
#define MLD_PHI2_L0 (2.885389949e+00f)
#define MLD_PHI2_L1 (9.618480019e-01f)
#define MLD_PHI2_L2 (5.740022860e-01f)
#define MLD_PHI2_L3 (4.702612714e-01f)
// base-2 fit '2H': max |small fit error| 5.39e-06 (bits), max relative large fit error 2.78e-06
#define MLD_PHI2H_S0 (-5.776050832e-02f)
#define MLD_PHI2H_S1 (1.608909580e-03f)
#define MLD_PHI2H_S2 (-4.610899829e-05f)
#define MLD_PHI2H_L0 (2.885398074e+00f)
#define MLD_PHI2H_L1 (9.600657329e-01f)
#define MLD_PHI2H_L2 (6.319043797e-01f)
