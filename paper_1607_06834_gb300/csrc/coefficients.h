// Method coefficients (binary64) of the ROK4 step, the classical RK4
// comparator and the ESDIRK3 comparator, shared by the single-problem and the
// batched drivers.
#pragma once

namespace rok {

// ROK4: alpha and b are the classical RK4 tableau; gamma is the L-stable root
// 0.5728160624821349 of g^4 - 4g^3 + 3g^2 - 2g/3 + 1/24 = 0; the off-diagonal
// gamma_ij solve the ROK order-4 conditions for Krylov dimension M >= 4 (the
// classical Rosenbrock conditions with the [[tau,tau]] condition split into its
// alpha part, 1/12, and its gamma part, -g/3), with gamma_41 = 3/5.
inline constexpr double kRokGamma = 0.5728160624821349;
inline constexpr double kRokAlpha[4][4] = {{0.0, 0.0, 0.0, 0.0}, {0.5, 0.0, 0.0, 0.0}, {0.0, 0.5, 0.0, 0.0}, {0.0, 0.0, 1.0, 0.0}};
inline constexpr double kRokGammaOff[4][4] = {{0.0, 0.0, 0.0, 0.0},
                                   {0.025068629909359066, 0.0, 0.0, 0.0},
                                   {0.2477474325727758, -1.405913872491725, 0.0, 0.0},
                                   {0.6, -0.020369905583413464, -1.7503308492902152, 0.0}};
inline constexpr double kRokB[4] = {0.16666666666666666, 0.3333333333333333, 0.3333333333333333, 0.16666666666666666};

// classical RK4
inline constexpr double kRk4A[4][4] = {{0.0, 0.0, 0.0, 0.0}, {0.5, 0.0, 0.0, 0.0}, {0.0, 0.5, 0.0, 0.0}, {0.0, 0.0, 1.0, 0.0}};
inline constexpr double kRk4B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

// ESDIRK3: explicit first stage, stage order 2, stiffly accurate, L-stable
// (gamma the root in (0.4, 0.5) of 6g^3 - 18g^2 + 9g - 1 = 0, c = (0, 2g, 3/5, 1)).
inline constexpr double kEsdGamma = 0.435866521508459;
inline constexpr double kEsdA[4][4] = {{0.0, 0.0, 0.0, 0.0},
                            {0.435866521508459, 0.435866521508459, 0.0, 0.0},
                            {0.2576482460664272, -0.09351476757488625, 0.435866521508459, 0.0},
                            {0.18764102434672383, -0.595297473576955, 0.9717899277217721, 0.435866521508459}};
inline constexpr double kEsdB[4] = {0.18764102434672383, -0.595297473576955, 0.9717899277217721, 0.435866521508459};

// embedded ROK4 weights (order 2 for every Krylov dimension, bhat_4 = 0): the error
// estimate of an adaptive step is sum_i (b_i - bhat_i) k_i
inline constexpr double kRokBhat[4] = {0.0, 0.4947033707526526, 0.5052966292473474, 0.0};

// DOPRI5 comparator: the Dormand-Prince 5(4) pair (J. Comput. Appl. Math. 6, 1980),
// 7 stages, first same as last (row 7 of A = b)
inline constexpr double kDp5A[7][7] = {
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0.0, 0.0, 0.0, 0.0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0.0, 0.0, 0.0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0.0, 0.0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0}};
inline constexpr double kDp5B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0,
                                    0.0};
inline constexpr double kDp5Bhat[7] = {5179.0 / 57600.0,    0.0,  7571.0 / 16695.0, 393.0 / 640.0,
                                       -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

// ROS4: the L-stable 4-stage Rosenbrock method of order 4 of Hairer & Wanner
// (Solving ODEs II, Sec. IV.7, g = 0.57282), published for the transformed
// stages u_i (implementation form (1/(h g) I - J) u_i = f(y + sum a_ij u_j)
// + sum (c_ij / h) u_j, y_1 = y_0 + sum m_j u_j); the driver converts it to
// the form of Eq. ROS (Sec. 2.2).
inline constexpr double kRos4Gamma = 0.57282;
inline constexpr double kRos4A[4][4] = {{0.0, 0.0, 0.0, 0.0},
                                        {2.000000000000000, 0.0, 0.0, 0.0},
                                        {1.867943637803922, 0.2344449711399156, 0.0, 0.0},
                                        {1.867943637803922, 0.2344449711399156, 0.0, 0.0}};
inline constexpr double kRos4C[4][4] = {{0.0, 0.0, 0.0, 0.0},
                                        {-7.137615036412310, 0.0, 0.0, 0.0},
                                        {2.580708087951457, 0.6515950076447975, 0.0, 0.0},
                                        {-2.137148994382534, -0.3214669691237626, -0.6949742501781779, 0.0}};
inline constexpr double kRos4M[4] = {2.255570073418735, 0.2870493262186792, 0.4353179431840180, 1.093502252409163};

// ROW: ROS34PW2 of Rang & Angermann (BIT 45, 2005), a 4-stage Rosenbrock-W
// method of order 3, L-stable, published in the form of Eq. ROS
// (g = 0.43586652150845900, the root of 6g^3 - 18g^2 + 9g - 1 in (0.4, 0.5)).
inline constexpr double kRowGamma = 0.43586652150845900;
inline constexpr double kRowAlpha[4][4] = {{0.0, 0.0, 0.0, 0.0},
                                           {0.87173304301691801, 0.0, 0.0, 0.0},
                                           {0.84457060015369423, -0.11299064236484185, 0.0, 0.0},
                                           {0.0, 0.0, 1.0, 0.0}};
inline constexpr double kRowGammaOff[4][4] = {{0.0, 0.0, 0.0, 0.0},
                                              {-0.87173304301691801, 0.0, 0.0, 0.0},
                                              {-0.90338057013044082, 0.054180672388095326, 0.0, 0.0},
                                              {0.24212380706095346, -1.2232505839045147, 0.54526025533510214, 0.0}};
inline constexpr double kRowB[4] = {0.24212380706095346, -1.2232505839045147, 1.5452602553351020,
                                    0.43586652150845900};

}  // namespace rok
