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
// fit 'H': max |small fit error| 3.73e-06, max relative large fit error 2.78e-06
#define MLD_PHIH_S0 (-8.333079853e-02f)
#define MLD_PHIH_S1 (4.831201677e-03f)
#define MLD_PHIH_S2 (-2.881758838e-04f)
#define MLD_PHIH_L0 (2.000005540e+00f)
#define MLD_PHIH_L1 (6.654668559e-01f)
#define MLD_PHIH_L2 (4.380027392e-01f)
