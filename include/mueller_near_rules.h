/*
 * mueller_near_rules.h -- near-panel quadrature data of the Nystrom
 * discretisation (Section 5), written by paper_1810_07067_gb300/near_rules.py.
 *
 * MUELLER_SELF_U / MUELLER_SELF_W: the generalized Gaussian rule on [0, 1]
 * with MUELLER_SELF_SIDE nodes that integrates Pt_j(u) and Pt_j(u) log u,
 * j < MUELLER_SELF_SIDE (Pt_j the Legendre polynomials shifted to [0, 1]),
 * exactly.  The target's own panel is split at the target and each side
 * mapped onto [0, 1] (u = distance from the target / side length), so the
 * pair of sides integrates p(t) log|t - t_i| + q(t), deg p, q < 16, exactly
 * (Remark after eq. eq_nyslike).  Values are the 60-digit solution rounded
 * to double.
 */
#ifndef MUELLER_NEAR_RULES_H
#define MUELLER_NEAR_RULES_H
#define MUELLER_SELF_SIDE 16
static const double MUELLER_SELF_U[MUELLER_SELF_SIDE] = {
  8.277309234714502e-05,
  0.0012283757008173626,
  0.0059798715382018705,
  0.018073696699772948,
  0.0417672109064258,
  0.08103861272100588,
  0.1387787920651679,
  0.21609636938067214,
  0.31184282304458977,
  0.4224350419037976,
  0.5420119053274876,
  0.6629152260330544,
  0.7764400251249938,
  0.8737610371066735,
  0.9469174698312383,
  0.9897391882007426,
};
static const double MUELLER_SELF_W[MUELLER_SELF_SIDE] = {
  0.00031563510123328075,
  0.0024060271597610428,
  0.0077311486995085,
  0.01717968538296474,
  0.030884140854647815,
  0.04815232117974444,
  0.06752091080786918,
  0.08692587041361871,
  0.10396721868051911,
  0.1162322159076941,
  0.12163241491114929,
  0.11870766643887921,
  0.10685433735889731,
  0.08644529923711167,
  0.05882560951438403,
  0.026219498352017572,
};
#endif
