// Generated by gen_erfcx_coef.py: erfcx(y) = exp(y^2) erfc(y) on 0 <= y <= 10 as a
// polynomial of degree 20 in s = (2 Z - Zmin - 1) / (1 - Zmin), Z = (L - y) / (L + y),
// L = 4.0, Zmin = (L - 10) / (L + 10); coefficient k as an FP32 pair (hi, lo).
// Largest relative error of the polynomial on 4001 points: 1.70e-17.
#pragma once

namespace gks {
namespace dfm {

constexpr float kErfcxL = 4.0f;
constexpr int kErfcxDeg = 20;
constexpr float kErfcxZminHi = -0.4285714328289032f, kErfcxZminLo = 4.257474817137563e-09f;
constexpr float kErfcxScaleHi = 1.399999976158142f, kErfcxScaleLo = 2.3841858265427618e-08f;
__device__ constexpr float kErfcxHi[kErfcxDeg + 1] = {
    0.2335701435804367f,
    0.31211239099502563f,
    0.2200557142496109f,
    0.13060057163238525f,
    0.06507864594459534f,
    0.026908960193395615f,
    0.008994290605187416f,
    0.0022964617237448692f,
    0.00038396770833060145f,
    1.3910656889493112e-05f,
    -1.2387361493892968e-05f,
    -2.9218906547612278e-06f,
    1.1467546556787056e-07f,
    1.5802324071501062e-07f,
    1.046868103316001e-08f,
    -7.67531638246055e-09f,
    -1.0318255139196708e-09f,
    3.949491567123431e-10f,
    6.790529943900836e-11f,
    -1.793206728939456e-11f,
    -3.1373035679765904e-12f};
__device__ constexpr float kErfcxLo[kErfcxDeg + 1] = {
    -2.7833144677913424e-09f,
    -1.2184431241735183e-08f,
    -2.364870521631701e-09f,
    -7.392558565300078e-09f,
    2.4001129972361923e-09f,
    -9.305551884608576e-10f,
    2.2101469265844997e-10f,
    9.971611730774654e-11f,
    -5.167100254610535e-12f,
    2.395914955148626e-13f,
    3.788996568755698e-13f,
    -4.7853373688752296e-14f,
    9.496444243088176e-16f,
    -2.0219127496004562e-15f,
    -2.461665150760577e-16f,
    -7.160608086573492e-17f,
    -1.0167039243084477e-18f,
    -5.86354380474696e-18f,
    -3.124179696322449e-18f,
    7.8282243181941215e-19f,
    -7.104870769893896e-20f};

}  // namespace dfm
}  // namespace gks
