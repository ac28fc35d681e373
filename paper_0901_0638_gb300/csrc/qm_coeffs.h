// Generated by paper_0901_0638_gb300/fit/gen_coeffs.py -- do not edit.
// Minimax rationals P(v)/Q(v) (monomial coefficients, constant term
// first) of the normal quantile in the paper's transformed coordinates;
// the generator's docstring gives each function, interval and degree.
#pragma once

#ifndef QM_COEF
#define QM_COEF static __constant__ const
#endif

namespace qm {
namespace coef {

// F64_EXP: [0, 42], degree (13,13); minimax relative error 5.38e-17, 1.24e-16 with double coefficients.
static constexpr double F64_EXP_LO = 0;
static constexpr double F64_EXP_HI = 42;
QM_COEF double F64_EXP_P[14] = {
    1.2533141373155001,
    6.066272156056464,
    11.918449262670602,
    12.334820485740778,
    7.332389193940919,
    2.5769271465297443,
    0.5356321100021414,
    0.0646666607697516,
    0.00438272646555109,
    0.0001581136628873452,
    2.7942607374112886e-06,
    2.10103400094353e-08,
    5.0655199730694676e-11,
    1.6473524355074186e-14};
QM_COEF double F64_EXP_Q[14] = {
    1.0,
    5.34018489494574,
    11.75117304840582,
    13.863627146317581,
    9.587314063383888,
    4.010833603056371,
    1.0180490672119398,
    0.1544059139676596,
    0.013579066429895894,
    0.0006613570875648861,
    1.6656795915644506e-05,
    1.9460951495759087e-07,
    8.675383161107495e-10,
    9.37483218411563e-13};

// F64_DEEP: [42, 745], degree (11,11); minimax relative error 9.9e-18, 5.69e-17 with double coefficients.
static constexpr double F64_DEEP_LO = 42;
static constexpr double F64_DEEP_HI = 745;
QM_COEF double F64_DEEP_P[12] = {
    1.1869349766480526,
    0.52878766978982,
    0.061426856950266194,
    0.0027162772879431502,
    5.347453752176976e-05,
    5.042152565399094e-07,
    2.336589782587857e-09,
    5.259779822648342e-12,
    5.450138634774207e-15,
    2.305227202713947e-18,
    3.0436789923309295e-22,
    5.331939614913202e-27};
QM_COEF double F64_DEEP_Q[12] = {
    1.0,
    0.8272771530263221,
    0.15746478289349505,
    0.010564767783888405,
    0.00030234318125367825,
    4.059007570007743e-06,
    2.6677215968468203e-08,
    8.62512873783402e-11,
    1.3283565761001979e-13,
    8.973647135894922e-17,
    2.2282936785087053e-20,
    1.3093034571754966e-24};

// F64_T2: [0, 15.5], degree (14,15); minimax relative error 5.21e-17, 1.04e-16 with double coefficients.
static constexpr double F64_T2_LO = 0;
static constexpr double F64_T2_HI = 15.5;
QM_COEF double F64_T2_P[15] = {
    1.2533141373155001,
    3.8044926829849173,
    8.256029905505297,
    12.416081397854986,
    14.639190014590403,
    13.516125942597235,
    9.907974924734923,
    5.655812151210451,
    2.430998804784557,
    0.7321431990703772,
    0.1339091187588571,
    0.012328237510453872,
    0.00048211641941322127,
    6.4400570114011425e-06,
    1.7819528822172512e-08};
QM_COEF double F64_T2_Q[16] = {
    1.0,
    3.035545973441099,
    6.82555940733442,
    10.629668562072073,
    13.180003479925036,
    12.933116699356834,
    10.267089099908116,
    6.50590059363855,
    3.2315513746422058,
    1.2039231264305694,
    0.3111440786373776,
    0.048413872305637214,
    0.00381868704968305,
    0.00012918139667906475,
    1.4887729370100395e-06,
    3.4097847664157757e-09};

// F32_PAPER: [0, 25], degree (5,6); minimax relative error 2.88e-08, 5.03e-08 with float coefficients.
static constexpr float F32_PAPER_LO = 0;
static constexpr float F32_PAPER_HI = 25;
QM_COEF float F32_PAPER_P[6] = {
    2.2616005e+00f,
    4.3491225e+00f,
    2.4086545e+00f,
    4.2863804e-01f,
    2.1474503e-02f,
    1.9942438e-04f};
QM_COEF float F32_PAPER_Q[7] = {
    1.8044962e+00f,
    4.3723407e+00f,
    3.3349106e+00f,
    9.193925e-01f,
    8.3534725e-02f,
    1.9091311e-03f,
    4.6910236e-06f};

// F32_SQRT: [0, 25], degree (6,6); minimax relative error 1.22e-09, 2.38e-08 with float coefficients.
static constexpr float F32_SQRT_LO = 0;
static constexpr float F32_SQRT_HI = 25;
QM_COEF float F32_SQRT_P[7] = {
    1.8187056e+00f,
    4.1437097e+00f,
    2.9659934e+00f,
    7.722647e-01f,
    6.7013875e-02f,
    1.4070297e-03f,
    2.0328443e-08f};
QM_COEF float F32_SQRT_Q[7] = {
    1.1578239e+00f,
    3.7957911e+00f,
    4.402373e+00f,
    2.194221e+00f,
    4.6194562e-01f,
    3.5627887e-02f,
    7.067321e-04f};

// F32_TAIL: [25, 104], degree (3,3); minimax relative error 5.46e-09, 3.49e-08 with float coefficients.
static constexpr float F32_TAIL_LO = 25;
static constexpr float F32_TAIL_HI = 104;
QM_COEF float F32_TAIL_P[4] = {
    2.732238e+00f,
    3.3398548e-01f,
    4.3988354e-03f,
    9.553332e-09f};
QM_COEF float F32_TAIL_Q[4] = {
    1.992515e+00f,
    1.7527925e+00f,
    1.7435963e-01f,
    2.2037574e-03f};

// F32_DEEP: [104, 745], degree (3,3); minimax relative error 1.2e-08, 3.43e-08 with float coefficients.
static constexpr float F32_DEEP_LO = 104;
static constexpr float F32_DEEP_HI = 745;
QM_COEF float F32_DEEP_P[4] = {
    1.7184582e+00f,
    4.8779093e-02f,
    1.3158191e-04f,
    9.9117485e-12f};
QM_COEF float F32_DEEP_Q[4] = {
    1.5921081e+00f,
    9.324607e-01f,
    2.4662642e-02f,
    6.5815846e-05f};

}  // namespace coef
}  // namespace qm
