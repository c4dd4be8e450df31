// masw_df.cuh -- the element stiffness in double-float arithmetic on the
// FP32 pipe, for the FP64 recurrence of the counting plan's certificate.
//
// GB300 issues 1.68 FP64 FMAs per clock per SM (measured) against 128 FP32
// FMAs, and an FP64 layer-evaluation (element + Schur step) takes about 98
// FP64 instructions, 29 of them the Schur step. Here the element's 4x4
// stiffness is computed with each value held as the unevaluated sum of two
// floats (hi + lo, |lo| <= ulp(hi)/2, a 48-bit significand: "double-float",
// after Dekker 1971 and the error-free sums and products of Knuth; products
// in the FMA form), converted to doubles exactly, and the Schur step of the
// recurrence stays in FP64 (masw_device.cuh::schur_layer). Inertia and sign
// decisions are the FP64 recurrence's.
//
// Accuracy. Below a layer's shear speed (r, s real) the element is written
// without cancellation: the rearrangement of the FP32 screen
// (masw_screen.cuh) for D, A1, D1, B1 and F1, and, for the coupling
// numerators, with sinh x_r - sinh x_s = 2 cosh((x_r+x_s)/2) sinh((x_r-x_s)/2),
//   E1 s = dS - (1 - rs) E_s h_r,   G1 r = -((1 - rs) E_r h_s + dS),
//   dS = (E_s - E_r)(1 + E_r E_s) / 2 = exp(-x_r-x_s)(sinh x_r - sinh x_s),
// (h_w = exp(-x_w) sinh x_w, E_w = exp(-x_w)), so its entries carry ~1e-13
// relative error where the plain FP64 forms lose digits to cancellation at
// low c. Above the shear speed the plain forms of masw_device.cuh are used
// (no such cancellation there), with ~1e-14 typical error.
//
// Functions: e^-x by a 256-entry table of 2^(j/256) and a degree-4 Taylor
// polynomial after the reduction x = (256 m + j) ln2/256 + r (Tang's method,
// with ln2/256 split in three floats so that n ln2/256 is exact to 48 bits);
// e^y - 1 for -0.35 < y <= 0 from (2^(-i/256) - 1) + 2^(-i/256)(e^r - 1),
// with no cancellation; 1/sqrt and 1/x by one Newton step from the SFU's
// float result; cosh - 1 and sinh/x by their Taylor series (high-order terms
// in float, where their error is below 2^-48 of the sum). Above the shear
// speed with both waves in the series (a layer thin next to the wavelength)
// the element's differences of cosh values near 1 are taken as differences of
// cosh - 1 instead. The trigonometric
// functions (layers slower than c with k h |w| > 1: about 1 % of the
// certificate's layer evaluations) run in FP64 and are split.
#pragma once

#include <cuda_runtime.h>

#include "masw_device.cuh"

namespace masw {

// ---------------------------------------------------------------- constants
// Written by gen_df_tables.py from 60-digit values; checked by
// tests/test_df_tables.py.
__device__ const float2 EXP2_DF[256] = {
    {0x1.0000000000000p+0f, 0x0.0p+0f}, {0x1.00b1b00000000p+0f, -0x1.6950d00000000p-26f},
    {0x1.0163da0000000p+0f, 0x1.3f66660000000p-25f}, {0x1.0216820000000p+0f, -0x1.789fb00000000p-25f},
    {0x1.02c9a40000000p+0f, -0x1.887fa00000000p-28f}, {0x1.037d420000000p+0f, 0x1.c2377a0000000p-25f},
    {0x1.04315e0000000p+0f, 0x1.0dcff00000000p-25f}, {0x1.04e5f80000000p+0f, -0x1.a1356a0000000p-25f},
    {0x1.059b0e0000000p+0f, -0x1.9d4f520000000p-25f}, {0x1.0650a00000000p+0f, 0x1.c783f20000000p-25f},
    {0x1.0706b20000000p+0f, 0x1.3bbedc0000000p-25f}, {0x1.07bd420000000p+0f, 0x1.6e55060000000p-25f},
    {0x1.0874520000000p+0f, -0x1.e2990e0000000p-26f}, {0x1.092be00000000p+0f, -0x1.333f040000000p-25f},
    {0x1.09e3ec0000000p+0f, 0x1.58de700000000p-25f}, {0x1.0a9c7a0000000p+0f, -0x1.3831ba0000000p-26f},
    {0x1.0b55860000000p+0f, 0x1.9f31220000000p-25f}, {0x1.0c0f140000000p+0f, 0x1.791b220000000p-26f},
    {0x1.0cc9220000000p+0f, 0x1.6e48fe0000000p-25f}, {0x1.0d83b20000000p+0f, 0x1.9caef60000000p-27f},
    {0x1.0e3ec40000000p+0f, -0x1.a585cc0000000p-25f}, {0x1.0efa560000000p+0f, -0x1.02b1da0000000p-31f},
    {0x1.0fb66a0000000p+0f, 0x1.ffda640000000p-25f}, {0x1.1073020000000p+0f, 0x1.1ae4680000000p-25f},
    {0x1.11301e0000000p+0f, -0x1.fdb4960000000p-25f}, {0x1.11edba0000000p+0f, 0x1.6bc5560000000p-25f},
    {0x1.12abdc0000000p+0f, 0x1.b0c7300000000p-30f}, {0x1.136a820000000p+0f, -0x1.61bf6a0000000p-25f},
    {0x1.1429aa0000000p+0f, 0x1.d525bc0000000p-25f}, {0x1.14e95a0000000p+0f, -0x1.9619da0000000p-25f},
    {0x1.15a98c0000000p+0f, 0x1.14b1ca0000000p-25f}, {0x1.166a460000000p+0f, -0x1.71c7880000000p-25f},
    {0x1.172b840000000p+0f, -0x1.c157420000000p-27f}, {0x1.17ed480000000p+0f, 0x1.a56ef00000000p-26f},
    {0x1.18af940000000p+0f, -0x1.dcdc860000000p-26f}, {0x1.1972660000000p+0f, -0x1.f228b40000000p-26f},
    {0x1.1a35be0000000p+0f, 0x1.6df96e0000000p-25f}, {0x1.1af9a00000000p+0f, -0x1.fb1d780000000p-26f},
    {0x1.1bbe080000000p+0f, 0x1.0117340000000p-26f}, {0x1.1c82fa0000000p+0f, -0x1.5afc720000000p-25f},
    {0x1.1d48740000000p+0f, -0x1.d2e8ca0000000p-25f}, {0x1.1e0e760000000p+0f, -0x1.4bbfda0000000p-28f},
    {0x1.1ed5020000000p+0f, 0x1.7e6c8e0000000p-27f}, {0x1.1f9c180000000p+0f, 0x1.0e33940000000p-26f},
    {0x1.2063b80000000p+0f, 0x1.0c519a0000000p-25f}, {0x1.212be40000000p+0f, -0x1.50eafc0000000p-25f},
    {0x1.21f49a0000000p+0f, -0x1.d0446e0000000p-25f}, {0x1.22bdda0000000p+0f, 0x1.3c89680000000p-27f},
    {0x1.2387a60000000p+0f, 0x1.ceac480000000p-25f}, {0x1.2452000000000p+0f, -0x1.1f7afe0000000p-26f},
    {0x1.251ce40000000p+0f, 0x1.f654c80000000p-25f}, {0x1.25e8580000000p+0f, -0x1.dc26320000000p-25f},
    {0x1.26b4560000000p+0f, 0x1.789f380000000p-26f}, {0x1.2780e40000000p+0f, -0x1.7c441a0000000p-25f},
    {0x1.284dfe0000000p+0f, 0x1.f563800000000p-28f}, {0x1.291ba80000000p+0f, -0x1.4dc8920000000p-25f},
    {0x1.29e9e00000000p+0f, -0x1.5c04240000000p-25f}, {0x1.2ab8a60000000p+0f, 0x1.b443c40000000p-26f},
    {0x1.2b87fe0000000p+0f, -0x1.e4a4ce0000000p-25f}, {0x1.2c57e40000000p+0f, -0x1.a239340000000p-26f},
    {0x1.2d285a0000000p+0f, 0x1.b900c20000000p-26f}, {0x1.2df9620000000p+0f, -0x1.37d4ee0000000p-29f},
    {0x1.2ecafa0000000p+0f, 0x1.27c5ea0000000p-25f}, {0x1.2f9d240000000p+0f, 0x1.57b10e0000000p-25f},
    {0x1.306fe00000000p+0f, 0x1.4636e20000000p-25f}, {0x1.31432e0000000p+0f, 0x1.bdd6600000000p-25f},
    {0x1.3217100000000p+0f, -0x1.d993e80000000p-27f}, {0x1.32eb840000000p+0f, -0x1.15c5740000000p-26f},
    {0x1.33c08c0000000p+0f, -0x1.b37d200000000p-25f}, {0x1.3496260000000p+0f, 0x1.b8fe8c0000000p-26f},
    {0x1.356c560000000p+0f, -0x1.b5803c0000000p-30f}, {0x1.36431a0000000p+0f, 0x1.6f441e0000000p-27f},
    {0x1.371a740000000p+0f, -0x1.18aac60000000p-25f}, {0x1.37f2620000000p+0f, 0x1.8f3aa40000000p-27f},
    {0x1.38cae60000000p+0f, 0x1.a0bb0c0000000p-25f}, {0x1.39a4020000000p+0f, -0x1.23afc40000000p-26f},
    {0x1.3a7db40000000p+0f, -0x1.634c020000000p-25f}, {0x1.3b57fc0000000p+0f, -0x1.3930ba0000000p-32f},
    {0x1.3c32dc0000000p+0f, 0x1.89d4720000000p-27f}, {0x1.3d0e540000000p+0f, 0x1.3b785c0000000p-26f},
    {0x1.3dea640000000p+0f, 0x1.8246840000000p-25f}, {0x1.3ec70e0000000p+0f, -0x1.c75d160000000p-29f},
    {0x1.3fa4500000000p+0f, 0x1.2b20060000000p-26f}, {0x1.40822c0000000p+0f, 0x1.b3d0120000000p-27f},
    {0x1.4160a20000000p+0f, 0x1.f72e2a0000000p-28f}, {0x1.423fb20000000p+0f, 0x1.c251a20000000p-26f},
    {0x1.431f5e0000000p+0f, -0x1.abd5da0000000p-26f}, {0x1.43ffa40000000p+0f, -0x1.ed18b00000000p-30f},
    {0x1.44e0860000000p+0f, 0x1.8624b40000000p-30f}, {0x1.45c2040000000p+0f, 0x1.53e9180000000p-27f},
    {0x1.46a41e0000000p+0f, 0x1.a3a00a0000000p-25f}, {0x1.4786d60000000p+0f, 0x1.a2cc8e0000000p-26f},
    {0x1.486a2c0000000p+0f, -0x1.47d8660000000p-25f}, {0x1.494e1e0000000p+0f, 0x1.92aed20000000p-28f},
    {0x1.4a32b00000000p+0f, -0x1.e505840000000p-25f}, {0x1.4b17de0000000p+0f, 0x1.4db6fa0000000p-25f},
    {0x1.4bfdae0000000p+0f, -0x1.593abc0000000p-25f}, {0x1.4ce41c0000000p+0f, -0x1.fa0fba0000000p-26f},
    {0x1.4dcb2a0000000p+0f, -0x1.8088bc0000000p-26f}, {0x1.4eb2d80000000p+0f, 0x1.d8abfe0000000p-28f},
    {0x1.4f9b280000000p+0f, -0x1.2c5a6c0000000p-25f}, {0x1.5084180000000p+0f, -0x1.759c240000000p-29f},
    {0x1.516daa0000000p+0f, 0x1.67b3200000000p-27f}, {0x1.5257de0000000p+0f, 0x1.07e9de0000000p-25f},
    {0x1.5342b60000000p+0f, -0x1.2c56100000000p-25f}, {0x1.542e300000000p+0f, -0x1.612a5c0000000p-25f},
    {0x1.551a4c0000000p+0f, 0x1.4bb2420000000p-25f}, {0x1.56070e0000000p+0f, -0x1.0b77980000000p-27f},
    {0x1.56f4740000000p+0f, -0x1.295b040000000p-25f}, {0x1.57e27e0000000p+0f, -0x1.074ecc0000000p-26f},
    {0x1.58d12e0000000p+0f, -0x1.6d07000000000p-25f}, {0x1.59c0820000000p+0f, 0x1.ffc1f20000000p-26f},
    {0x1.5ab07e0000000p+0f, -0x1.5bd5ec0000000p-27f}, {0x1.5ba1200000000p+0f, -0x1.15e1800000000p-26f},
    {0x1.5c92680000000p+0f, 0x1.4b28d60000000p-25f}, {0x1.5d845a0000000p+0f, -0x1.ecce8e0000000p-25f},
    {0x1.5e76f20000000p+0f, -0x1.4a5bd60000000p-25f}, {0x1.5f6a320000000p+0f, 0x1.b9d6e20000000p-29f},
    {0x1.605e1c0000000p+0f, -0x1.a248fe0000000p-26f}, {0x1.6152ae0000000p+0f, 0x1.b37dbe0000000p-26f},
    {0x1.6247ec0000000p+0f, -0x1.f8b5500000000p-25f}, {0x1.633dd20000000p+0f, -0x1.736b020000000p-27f},
    {0x1.6434640000000p+0f, -0x1.66679c0000000p-25f}, {0x1.652ba00000000p+0f, -0x1.43704a0000000p-28f},
    {0x1.6623880000000p+0f, 0x1.2a91120000000p-27f}, {0x1.671c1c0000000p+0f, 0x1.c20cfe0000000p-26f},
    {0x1.68155e0000000p+0f, -0x1.766ad20000000p-25f}, {0x1.690f4c0000000p+0f, -0x1.cc2d580000000p-25f},
    {0x1.6a09e60000000p+0f, 0x1.9fcef40000000p-26f}, {0x1.6b05300000000p+0f, -0x1.62ba300000000p-26f},
    {0x1.6c01280000000p+0f, -0x1.5e84a80000000p-25f}, {0x1.6cfdce0000000p+0f, -0x1.15c4de0000000p-27f},
    {0x1.6dfb240000000p+0f, -0x1.cd72e80000000p-27f}, {0x1.6ef92a0000000p+0f, -0x1.e9b1460000000p-26f},
    {0x1.6ff7e00000000p+0f, -0x1.ab9ae00000000p-26f}, {0x1.70f7460000000p+0f, 0x1.bd0ba20000000p-26f},
    {0x1.71f75e0000000p+0f, 0x1.1d8bee0000000p-25f}, {0x1.72f8280000000p+0f, 0x1.bab4220000000p-26f},
    {0x1.73f9a40000000p+0f, 0x1.14b02e0000000p-25f}, {0x1.74fbd40000000p+0f, -0x1.4506800000000p-25f},
    {0x1.75feb60000000p+0f, -0x1.37b3060000000p-25f}, {0x1.77024c0000000p+0f, -0x1.ca923e0000000p-25f},
    {0x1.7806940000000p+0f, 0x1.fbcba80000000p-25f}, {0x1.790b940000000p+0f, -0x1.d4f8c20000000p-26f},
    {0x1.7a11480000000p+0f, -0x1.829fd00000000p-25f}, {0x1.7b17b00000000p+0f, 0x1.2ed9fc0000000p-25f},
    {0x1.7c1ed00000000p+0f, 0x1.30c1320000000p-28f}, {0x1.7d26a60000000p+0f, 0x1.7fc3780000000p-27f},
    {0x1.7e2f340000000p+0f, -0x1.2616340000000p-25f}, {0x1.7f38780000000p+0f, 0x1.2471240000000p-26f},
    {0x1.8042760000000p+0f, -0x1.783cbe0000000p-25f}, {0x1.814d2a0000000p+0f, 0x1.ba20dc0000000p-25f},
    {0x1.82589a0000000p+0f, -0x1.accc7c0000000p-26f}, {0x1.8364c20000000p+0f, -0x1.46be080000000p-28f},
    {0x1.8471a40000000p+0f, 0x1.88f1ec0000000p-26f}, {0x1.857f420000000p+0f, -0x1.0c149c0000000p-25f},
    {0x1.868d9a0000000p+0f, -0x1.2edb440000000p-26f}, {0x1.879cae0000000p+0f, -0x1.b396f20000000p-26f},
    {0x1.88ac7e0000000p+0f, -0x1.9d665a0000000p-26f}, {0x1.89bd0a0000000p+0f, 0x1.1e16040000000p-26f},
    {0x1.8ace540000000p+0f, 0x1.15506e0000000p-27f}, {0x1.8be05c0000000p+0f, -0x1.4a7a220000000p-26f},
    {0x1.8cf3220000000p+0f, -0x1.29576e0000000p-25f}, {0x1.8e06a60000000p+0f, -0x1.f799280000000p-28f},
    {0x1.8f1aea0000000p+0f, -0x1.baa2320000000p-26f}, {0x1.902fee0000000p+0f, -0x1.fafa6e0000000p-25f},
    {0x1.9145b00000000p+0f, 0x1.723ff80000000p-25f}, {0x1.925c360000000p+0f, -0x1.8aba040000000p-25f},
    {0x1.93737c0000000p+0f, -0x1.e647440000000p-25f}, {0x1.948b820000000p+0f, 0x1.6bf31c0000000p-25f},
    {0x1.95a44c0000000p+0f, 0x1.790a420000000p-25f}, {0x1.96bdda0000000p+0f, -0x1.6263d40000000p-26f},
    {0x1.97d82a0000000p+0f, -0x1.0d8d840000000p-31f}, {0x1.98f33e0000000p+0f, 0x1.1e88a80000000p-26f},
    {0x1.9a0f180000000p+0f, -0x1.e6bf080000000p-25f}, {0x1.9b2bb40000000p+0f, 0x1.aa7fc20000000p-25f},
    {0x1.9c49180000000p+0f, 0x1.51f8480000000p-27f}, {0x1.9d67420000000p+0f, -0x1.ad11ca0000000p-26f},
    {0x1.9e86320000000p+0f, -0x1.8737380000000p-26f}, {0x1.9fa5e80000000p+0f, 0x1.a0fe540000000p-25f},
    {0x1.a0c6680000000p+0f, -0x1.2886a60000000p-26f}, {0x1.a1e7ae0000000p+0f, 0x1.b1d7180000000p-25f},
    {0x1.a309be0000000p+0f, 0x1.8945a60000000p-25f}, {0x1.a42c980000000p+0f, 0x1.182b5e0000000p-30f},
    {0x1.a5503c0000000p+0f, -0x1.b83b540000000p-25f}, {0x1.a674a80000000p+0f, 0x1.5e8c0a0000000p-25f},
    {0x1.a799e20000000p+0f, -0x1.99e9940000000p-25f}, {0x1.a8bfe60000000p+0f, -0x1.87da340000000p-25f},
    {0x1.a9e6b60000000p+0f, -0x1.50c0480000000p-25f}, {0x1.ab0e520000000p+0f, 0x1.356eba0000000p-28f},
    {0x1.ac36bc0000000p+0f, -0x1.6064320000000p-31f}, {0x1.ad5ff40000000p+0f, -0x1.70f6220000000p-26f},
    {0x1.ae89fa0000000p+0f, -0x1.a94b140000000p-26f}, {0x1.afb4ce0000000p+0f, 0x1.88bcc00000000p-26f},
    {0x1.b0e0720000000p+0f, 0x1.31b6cc0000000p-25f}, {0x1.b20ce60000000p+0f, 0x1.93512a0000000p-25f},
    {0x1.b33a2c0000000p+0f, -0x1.ec3a820000000p-26f}, {0x1.b468420000000p+0f, -0x1.4916ca0000000p-25f},
    {0x1.b597280000000p+0f, 0x1.bcab280000000p-25f}, {0x1.b6c6e20000000p+0f, 0x1.3e38a60000000p-25f},
    {0x1.b7f7700000000p+0f, -0x1.a094380000000p-25f}, {0x1.b928d00000000p+0f, -0x1.bb16c40000000p-25f},
    {0x1.ba5b040000000p+0f, -0x1.ebdf360000000p-25f}, {0x1.bb8e0c0000000p+0f, -0x1.0cb21c0000000p-25f},
    {0x1.bcc1ea0000000p+0f, -0x1.f687c60000000p-25f}, {0x1.bdf69c0000000p+0f, 0x1.f9d1040000000p-27f},
    {0x1.bf2c260000000p+0f, -0x1.0a387e0000000p-26f}, {0x1.c062860000000p+0f, 0x1.41b33c0000000p-28f},
    {0x1.c199be0000000p+0f, -0x1.3d56b20000000p-27f}, {0x1.c2d1ce0000000p+0f, -0x1.8166b60000000p-26f},
    {0x1.c40ab60000000p+0f, -0x1.7c2c980000000p-39f}, {0x1.c544780000000p+0f, -0x1.c141380000000p-26f},
    {0x1.c67f120000000p+0f, 0x1.cafa2a0000000p-25f}, {0x1.c7ba880000000p+0f, 0x1.3119260000000p-25f},
    {0x1.c8f6da0000000p+0f, -0x1.7f230a0000000p-25f}, {0x1.ca34060000000p+0f, -0x1.15c7640000000p-25f},
    {0x1.cb720e0000000p+0f, -0x1.8837cc0000000p-27f}, {0x1.ccb0f20000000p+0f, 0x1.cda2ce0000000p-25f},
    {0x1.cdf0b60000000p+0f, -0x1.5447800000000p-25f}, {0x1.cf31560000000p+0f, -0x1.2915240000000p-26f},
    {0x1.d072d40000000p+0f, 0x1.40f1300000000p-25f}, {0x1.d1b5320000000p+0f, 0x1.61192e0000000p-25f},
    {0x1.d2f8700000000p+0f, 0x1.01b13e0000000p-25f}, {0x1.d43c8e0000000p+0f, 0x1.59543a0000000p-25f},
    {0x1.d5818e0000000p+0f, -0x1.822dbc0000000p-27f}, {0x1.d6c76e0000000p+0f, 0x1.0c5cda0000000p-25f},
    {0x1.d80e320000000p+0f, -0x1.26cf8e0000000p-25f}, {0x1.d955d80000000p+0f, -0x1.c013f20000000p-25f},
    {0x1.da9e600000000p+0f, 0x1.ed99420000000p-27f}, {0x1.dbe7ce0000000p+0f, -0x1.38af9e0000000p-25f},
    {0x1.dd32200000000p+0f, -0x1.9fc9740000000p-25f}, {0x1.de7d560000000p+0f, 0x1.0701960000000p-26f},
    {0x1.dfc9740000000p+0f, -0x1.908c940000000p-25f}, {0x1.e116760000000p+0f, 0x1.632fa20000000p-25f},
    {0x1.e264620000000p+0f, -0x1.614bda0000000p-25f}, {0x1.e3b3340000000p+0f, -0x1.3a447c0000000p-26f},
    {0x1.e502ee0000000p+0f, 0x1.e2cffe0000000p-26f}, {0x1.e653920000000p+0f, 0x1.19db5e0000000p-26f},
    {0x1.e7a5200000000p+0f, -0x1.0e2ce00000000p-26f}, {0x1.e8f7980000000p+0f, -0x1.0649180000000p-25f},
    {0x1.ea4afa0000000p+0f, 0x1.52486c0000000p-27f}, {0x1.eb9f480000000p+0f, 0x1.9f329c0000000p-26f},
    {0x1.ecf4820000000p+0f, 0x1.b1ccfe0000000p-25f}, {0x1.ee4aaa0000000p+0f, 0x1.0c42880000000p-27f},
    {0x1.efa1be0000000p+0f, 0x1.cc2b440000000p-25f}, {0x1.f0f9c20000000p+0f, -0x1.a4df6c0000000p-27f},
    {0x1.f252b40000000p+0f, -0x1.1288ae0000000p-25f}, {0x1.f3ac940000000p+0f, 0x1.1bae4e0000000p-25f},
    {0x1.f507660000000p+0f, -0x1.246eb00000000p-26f}, {0x1.f663280000000p+0f, -0x1.9deec20000000p-26f},
    {0x1.f7bfda0000000p+0f, 0x1.b397c20000000p-25f}, {0x1.f91d800000000p+0f, 0x1.121e440000000p-27f},
    {0x1.fa7c180000000p+0f, 0x1.9e90d80000000p-28f}, {0x1.fbdba40000000p+0f, -0x1.2da55e0000000p-25f},
    {0x1.fd3c220000000p+0f, 0x1.71ee3e0000000p-25f}, {0x1.fe9d960000000p+0f, 0x1.65447c0000000p-25f},
};
__device__ const float2 EXPM1_DF[131] = {
    {0x0.0p+0f, 0x0.0p+0f}, {-0x1.62694e0000000p-9f, 0x1.447b220000000p-34f},
    {-0x1.61eea40000000p-8f, 0x1.ee3e220000000p-34f}, {-0x1.0917260000000p-7f, 0x1.2d513e0000000p-33f},
    {-0x1.60f9fa0000000p-7f, 0x1.e90d820000000p-33f}, {-0x1.b89ff80000000p-7f, 0x1.21e4480000000p-32f},
    {-0x1.0804a40000000p-6f, -0x1.8d07b20000000p-31f}, {-0x1.339b0c0000000p-6f, -0x1.deec1e0000000p-31f},
    {-0x1.5f134a0000000p-6f, 0x1.b915020000000p-31f}, {-0x1.8a6d6e0000000p-6f, -0x1.146c600000000p-32f},
    {-0x1.b5a9920000000p-6f, 0x1.aeea5e0000000p-31f}, {-0x1.e0c7c60000000p-6f, -0x1.26fb5a0000000p-31f},
    {-0x1.05e4120000000p-5f, 0x1.85689e0000000p-31f}, {-0x1.1b555e0000000p-5f, 0x1.8851040000000p-33f},
    {-0x1.30b7d20000000p-5f, -0x1.c6603e0000000p-31f}, {-0x1.460b7a0000000p-5f, 0x1.f329ba0000000p-31f},
    {-0x1.5b505e0000000p-5f, 0x1.4921b40000000p-30f}, {-0x1.7086880000000p-5f, -0x1.9246020000000p-32f},
    {-0x1.85ae040000000p-5f, -0x1.c59be60000000p-32f}, {-0x1.9ac6dc0000000p-5f, 0x1.9db5d80000000p-31f},
    {-0x1.afd1180000000p-5f, -0x1.d300280000000p-31f}, {-0x1.c4ccc40000000p-5f, -0x1.d223dc0000000p-30f},
    {-0x1.d9b9ec0000000p-5f, 0x1.eb42520000000p-30f}, {-0x1.ee98940000000p-5f, -0x1.cd05d20000000p-30f},
    {-0x1.01b4660000000p-4f, -0x1.08c9420000000p-30f}, {-0x1.0c154e0000000p-4f, 0x1.c065780000000p-33f},
    {-0x1.166f060000000p-4f, -0x1.fc97400000000p-30f}, {-0x1.20c1940000000p-4f, -0x1.c57cec0000000p-29f},
    {-0x1.2b0cfe0000000p-4f, -0x1.266bd40000000p-32f}, {-0x1.3551480000000p-4f, 0x1.ff60760000000p-29f},
    {-0x1.3f8e740000000p-4f, -0x1.367c680000000p-29f}, {-0x1.49c48c0000000p-4f, 0x1.8b9b4c0000000p-31f},
    {-0x1.53f3920000000p-4f, 0x1.f7490e0000000p-30f}, {-0x1.5e1b8a0000000p-4f, -0x1.355e2a0000000p-29f},
    {-0x1.683c7c0000000p-4f, 0x1.b13e320000000p-34f}, {-0x1.72566a0000000p-4f, -0x1.ee6d300000000p-30f},
    {-0x1.7c695a0000000p-4f, -0x1.f876840000000p-29f}, {-0x1.8675520000000p-4f, -0x1.48a9180000000p-30f},
    {-0x1.907a560000000p-4f, 0x1.5dc3fa0000000p-29f}, {-0x1.9a78680000000p-4f, -0x1.92e98c0000000p-29f},
    {-0x1.a46f920000000p-4f, 0x1.df20d20000000p-30f}, {-0x1.ae5fd40000000p-4f, -0x1.5c764a0000000p-30f},
    {-0x1.b849360000000p-4f, 0x1.b9ed440000000p-35f}, {-0x1.c22bbc0000000p-4f, 0x1.88c9320000000p-29f},
    {-0x1.cc07680000000p-4f, -0x1.a82eb40000000p-29f}, {-0x1.d5dc440000000p-4f, 0x1.f5f6440000000p-30f},
    {-0x1.dfaa500000000p-4f, -0x1.7c2c980000000p-40f}, {-0x1.e971940000000p-4f, 0x1.fa652c0000000p-29f},
    {-0x1.f332120000000p-4f, 0x1.85529c0000000p-29f}, {-0x1.fcebd00000000p-4f, 0x1.41b33c0000000p-29f},
    {-0x1.034f6a0000000p-3f, 0x1.eb8f040000000p-28f}, {-0x1.0825900000000p-3f, 0x1.f9d1040000000p-28f},
    {-0x1.0cf85c0000000p-3f, 0x1.2f07480000000p-31f}, {-0x1.11c7d20000000p-3f, -0x1.9643840000000p-31f},
    {-0x1.1693f40000000p-3f, 0x1.420c940000000p-30f}, {-0x1.1b5cc40000000p-3f, 0x1.13a4f20000000p-28f},
    {-0x1.2022440000000p-3f, 0x1.7daf240000000p-28f}, {-0x1.24e4760000000p-3f, 0x1.f1c52a0000000p-29f},
    {-0x1.29a35c0000000p-3f, -0x1.0d53640000000p-28f}, {-0x1.2e5efa0000000p-3f, -0x1.245b280000000p-28f},
    {-0x1.3317520000000p-3f, 0x1.3c57ec0000000p-31f}, {-0x1.37cc640000000p-3f, -0x1.b2bb560000000p-28f},
    {-0x1.3c7e360000000p-3f, 0x1.8db6660000000p-29f}, {-0x1.412cc60000000p-3f, -0x1.dd0d020000000p-29f},
    {-0x1.45d81a0000000p-3f, 0x1.5ad3ae0000000p-29f}, {-0x1.4a80320000000p-3f, 0x1.1e13ba0000000p-28f},
    {-0x1.4f25100000000p-3f, -0x1.6064320000000p-32f}, {-0x1.53c6b80000000p-3f, 0x1.356eba0000000p-29f},
    {-0x1.58652a0000000p-3f, -0x1.4301200000000p-28f}, {-0x1.5d006c0000000p-3f, 0x1.e0972c0000000p-28f},
    {-0x1.61987c0000000p-3f, 0x1.9859ac0000000p-28f}, {-0x1.662d5e0000000p-3f, 0x1.7a302a0000000p-28f},
    {-0x1.6abf140000000p-3f, 0x1.1f12ae0000000p-28f}, {-0x1.6f4da00000000p-3f, 0x1.182b5e0000000p-31f},
    {-0x1.73d9040000000p-3f, -0x1.dae9660000000p-28f}, {-0x1.7861440000000p-3f, -0x1.38a3a20000000p-28f},
    {-0x1.7ce6620000000p-3f, 0x1.aef2b20000000p-28f}, {-0x1.81685c0000000p-3f, -0x1.7c06b20000000p-28f},
    {-0x1.85e73a0000000p-3f, 0x1.e323240000000p-29f}, {-0x1.8a62fa0000000p-3f, 0x1.4bb8d40000000p-29f},
    {-0x1.8edba00000000p-3f, 0x1.51f8480000000p-28f}, {-0x1.93512c0000000p-3f, -0x1.5600fa0000000p-28f},
    {-0x1.97c3a40000000p-3f, 0x1.940f740000000p-30f}, {-0x1.9c33060000000p-3f, -0x1.c2eeae0000000p-28f},
    {-0x1.a09f580000000p-3f, -0x1.0d8d840000000p-32f}, {-0x1.a5089a0000000p-3f, 0x1.3b385a0000000p-28f},
    {-0x1.a96ece0000000p-3f, 0x1.e429080000000p-28f}, {-0x1.add1f60000000p-3f, 0x1.afcc720000000p-28f},
    {-0x1.b232140000000p-3f, 0x1.9b8bca0000000p-30f}, {-0x1.b68f2c0000000p-3f, 0x1.d517f00000000p-28f},
    {-0x1.bae93e0000000p-3f, 0x1.c8ffe20000000p-28f}, {-0x1.bf404c0000000p-3f, 0x1.4164520000000p-32f},
    {-0x1.c3945a0000000p-3f, 0x1.1577360000000p-29f}, {-0x1.c7e5680000000p-3f, -0x1.f799280000000p-29f},
    {-0x1.cc337a0000000p-3f, -0x1.4abb740000000p-29f}, {-0x1.d07e920000000p-3f, 0x1.6b0bbc0000000p-28f},
    {-0x1.d4c6b00000000p-3f, 0x1.15506e0000000p-28f}, {-0x1.d90bd60000000p-3f, -0x1.c3d3f80000000p-28f},
    {-0x1.dd4e0a0000000p-3f, 0x1.8a669a0000000p-29f}, {-0x1.e18d4a0000000p-3f, 0x1.31a4360000000p-29f},
    {-0x1.e5c99a0000000p-3f, 0x1.a249760000000p-28f}, {-0x1.ea02fa0000000p-3f, -0x1.82937c0000000p-31f},
    {-0x1.ee396e0000000p-3f, -0x1.dc38540000000p-29f}, {-0x1.f26cf80000000p-3f, -0x1.46be080000000p-29f},
    {-0x1.f69d9a0000000p-3f, 0x1.4cce120000000p-29f}, {-0x1.facb540000000p-3f, -0x1.177c940000000p-28f},
    {-0x1.fef62a0000000p-3f, -0x1.e0f2f80000000p-28f}, {-0x1.018f100000000p-2f, 0x1.2471240000000p-27f},
    {-0x1.03a19a0000000p-2f, 0x1.b3d3980000000p-27f}, {-0x1.05b2b40000000p-2f, 0x1.7fc3780000000p-28f},
    {-0x1.07c2600000000p-2f, 0x1.30c1320000000p-29f}, {-0x1.09d09e0000000p-2f, -0x1.a24c0a0000000p-27f},
    {-0x1.0bdd720000000p-2f, 0x1.f580c40000000p-28f}, {-0x1.0de8d80000000p-2f, -0x1.d4f8c20000000p-27f},
    {-0x1.0ff2d60000000p-2f, -0x1.0d16040000000p-32f}, {-0x1.11fb6a0000000p-2f, 0x1.ab6e0a0000000p-29f},
    {-0x1.1402960000000p-2f, 0x1.9099f20000000p-27f}, {-0x1.16085a0000000p-2f, 0x1.75f3000000000p-27f},
    {-0x1.180cb60000000p-2f, -0x1.d69fa40000000p-27f}, {-0x1.1a0fb00000000p-2f, 0x1.bab4220000000p-27f},
    {-0x1.1c11420000000p-2f, -0x1.c4e8240000000p-27f}, {-0x1.1e11740000000p-2f, 0x1.bd0ba20000000p-27f},
    {-0x1.2010400000000p-2f, -0x1.ab9ae00000000p-27f}, {-0x1.220dac0000000p-2f, -0x1.e9b1460000000p-27f},
    {-0x1.2409b80000000p-2f, -0x1.cd72e80000000p-28f}, {-0x1.2604640000000p-2f, -0x1.15c4de0000000p-28f},
    {-0x1.27fdb20000000p-2f, 0x1.42f6b00000000p-27f}, {-0x1.29f5a00000000p-2f, -0x1.62ba300000000p-27f},
    {-0x1.2bec340000000p-2f, 0x1.9fcef40000000p-27f}, {-0x1.2de16a0000000p-2f, 0x1.9e95380000000p-29f},
    {-0x1.2fd5460000000p-2f, 0x1.132a5c0000000p-27f},
};
__device__ const float2 EXP2N_DF[131] = {
    {0x1.0000000000000p+0f, 0x0.0p+0f}, {0x1.fe9d960000000p-1f, 0x1.65447c0000000p-26f},
    {0x1.fd3c220000000p-1f, 0x1.71ee3e0000000p-26f}, {0x1.fbdba40000000p-1f, -0x1.2da55e0000000p-26f},
    {0x1.fa7c180000000p-1f, 0x1.9e90d80000000p-29f}, {0x1.f91d800000000p-1f, 0x1.121e440000000p-28f},
    {0x1.f7bfda0000000p-1f, 0x1.b397c20000000p-26f}, {0x1.f663280000000p-1f, -0x1.9deec20000000p-27f},
    {0x1.f507660000000p-1f, -0x1.246eb00000000p-27f}, {0x1.f3ac940000000p-1f, 0x1.1bae4e0000000p-26f},
    {0x1.f252b40000000p-1f, -0x1.1288ae0000000p-26f}, {0x1.f0f9c20000000p-1f, -0x1.a4df6c0000000p-28f},
    {0x1.efa1be0000000p-1f, 0x1.cc2b440000000p-26f}, {0x1.ee4aaa0000000p-1f, 0x1.0c42880000000p-28f},
    {0x1.ecf4820000000p-1f, 0x1.b1ccfe0000000p-26f}, {0x1.eb9f480000000p-1f, 0x1.9f329c0000000p-27f},
    {0x1.ea4afa0000000p-1f, 0x1.52486c0000000p-28f}, {0x1.e8f7980000000p-1f, -0x1.0649180000000p-26f},
    {0x1.e7a5200000000p-1f, -0x1.0e2ce00000000p-27f}, {0x1.e653920000000p-1f, 0x1.19db5e0000000p-27f},
    {0x1.e502ee0000000p-1f, 0x1.e2cffe0000000p-27f}, {0x1.e3b3340000000p-1f, -0x1.3a447c0000000p-27f},
    {0x1.e264620000000p-1f, -0x1.614bda0000000p-26f}, {0x1.e116760000000p-1f, 0x1.632fa20000000p-26f},
    {0x1.dfc9740000000p-1f, -0x1.908c940000000p-26f}, {0x1.de7d560000000p-1f, 0x1.0701960000000p-27f},
    {0x1.dd32200000000p-1f, -0x1.9fc9740000000p-26f}, {0x1.dbe7ce0000000p-1f, -0x1.38af9e0000000p-26f},
    {0x1.da9e600000000p-1f, 0x1.ed99420000000p-28f}, {0x1.d955d80000000p-1f, -0x1.c013f20000000p-26f},
    {0x1.d80e320000000p-1f, -0x1.26cf8e0000000p-26f}, {0x1.d6c76e0000000p-1f, 0x1.0c5cda0000000p-26f},
    {0x1.d5818e0000000p-1f, -0x1.822dbc0000000p-28f}, {0x1.d43c8e0000000p-1f, 0x1.59543a0000000p-26f},
    {0x1.d2f8700000000p-1f, 0x1.01b13e0000000p-26f}, {0x1.d1b5320000000p-1f, 0x1.61192e0000000p-26f},
    {0x1.d072d40000000p-1f, 0x1.40f1300000000p-26f}, {0x1.cf31560000000p-1f, -0x1.2915240000000p-27f},
    {0x1.cdf0b60000000p-1f, -0x1.5447800000000p-26f}, {0x1.ccb0f20000000p-1f, 0x1.cda2ce0000000p-26f},
    {0x1.cb720e0000000p-1f, -0x1.8837cc0000000p-28f}, {0x1.ca34060000000p-1f, -0x1.15c7640000000p-26f},
    {0x1.c8f6da0000000p-1f, -0x1.7f230a0000000p-26f}, {0x1.c7ba880000000p-1f, 0x1.3119260000000p-26f},
    {0x1.c67f120000000p-1f, 0x1.cafa2a0000000p-26f}, {0x1.c544780000000p-1f, -0x1.c141380000000p-27f},
    {0x1.c40ab60000000p-1f, -0x1.7c2c980000000p-40f}, {0x1.c2d1ce0000000p-1f, -0x1.8166b60000000p-27f},
    {0x1.c199be0000000p-1f, -0x1.3d56b20000000p-28f}, {0x1.c062860000000p-1f, 0x1.41b33c0000000p-29f},
    {0x1.bf2c260000000p-1f, -0x1.0a387e0000000p-27f}, {0x1.bdf69c0000000p-1f, 0x1.f9d1040000000p-28f},
    {0x1.bcc1ea0000000p-1f, -0x1.f687c60000000p-26f}, {0x1.bb8e0c0000000p-1f, -0x1.0cb21c0000000p-26f},
    {0x1.ba5b040000000p-1f, -0x1.ebdf360000000p-26f}, {0x1.b928d00000000p-1f, -0x1.bb16c40000000p-26f},
    {0x1.b7f7700000000p-1f, -0x1.a094380000000p-26f}, {0x1.b6c6e20000000p-1f, 0x1.3e38a60000000p-26f},
    {0x1.b597280000000p-1f, 0x1.bcab280000000p-26f}, {0x1.b468420000000p-1f, -0x1.4916ca0000000p-26f},
    {0x1.b33a2c0000000p-1f, -0x1.ec3a820000000p-27f}, {0x1.b20ce60000000p-1f, 0x1.93512a0000000p-26f},
    {0x1.b0e0720000000p-1f, 0x1.31b6cc0000000p-26f}, {0x1.afb4ce0000000p-1f, 0x1.88bcc00000000p-27f},
    {0x1.ae89fa0000000p-1f, -0x1.a94b140000000p-27f}, {0x1.ad5ff40000000p-1f, -0x1.70f6220000000p-27f},
    {0x1.ac36bc0000000p-1f, -0x1.6064320000000p-32f}, {0x1.ab0e520000000p-1f, 0x1.356eba0000000p-29f},
    {0x1.a9e6b60000000p-1f, -0x1.50c0480000000p-26f}, {0x1.a8bfe60000000p-1f, -0x1.87da340000000p-26f},
    {0x1.a799e20000000p-1f, -0x1.99e9940000000p-26f}, {0x1.a674a80000000p-1f, 0x1.5e8c0a0000000p-26f},
    {0x1.a5503c0000000p-1f, -0x1.b83b540000000p-26f}, {0x1.a42c980000000p-1f, 0x1.182b5e0000000p-31f},
    {0x1.a309be0000000p-1f, 0x1.8945a60000000p-26f}, {0x1.a1e7ae0000000p-1f, 0x1.b1d7180000000p-26f},
    {0x1.a0c6680000000p-1f, -0x1.2886a60000000p-27f}, {0x1.9fa5e80000000p-1f, 0x1.a0fe540000000p-26f},
    {0x1.9e86320000000p-1f, -0x1.8737380000000p-27f}, {0x1.9d67420000000p-1f, -0x1.ad11ca0000000p-27f},
    {0x1.9c49180000000p-1f, 0x1.51f8480000000p-28f}, {0x1.9b2bb40000000p-1f, 0x1.aa7fc20000000p-26f},
    {0x1.9a0f180000000p-1f, -0x1.e6bf080000000p-26f}, {0x1.98f33e0000000p-1f, 0x1.1e88a80000000p-27f},
    {0x1.97d82a0000000p-1f, -0x1.0d8d840000000p-32f}, {0x1.96bdda0000000p-1f, -0x1.6263d40000000p-27f},
    {0x1.95a44c0000000p-1f, 0x1.790a420000000p-26f}, {0x1.948b820000000p-1f, 0x1.6bf31c0000000p-26f},
    {0x1.93737c0000000p-1f, -0x1.e647440000000p-26f}, {0x1.925c360000000p-1f, -0x1.8aba040000000p-26f},
    {0x1.9145b00000000p-1f, 0x1.723ff80000000p-26f}, {0x1.902fee0000000p-1f, -0x1.fafa6e0000000p-26f},
    {0x1.8f1aea0000000p-1f, -0x1.baa2320000000p-27f}, {0x1.8e06a60000000p-1f, -0x1.f799280000000p-29f},
    {0x1.8cf3220000000p-1f, -0x1.29576e0000000p-26f}, {0x1.8be05c0000000p-1f, -0x1.4a7a220000000p-27f},
    {0x1.8ace540000000p-1f, 0x1.15506e0000000p-28f}, {0x1.89bd0a0000000p-1f, 0x1.1e16040000000p-27f},
    {0x1.88ac7e0000000p-1f, -0x1.9d665a0000000p-27f}, {0x1.879cae0000000p-1f, -0x1.b396f20000000p-27f},
    {0x1.868d9a0000000p-1f, -0x1.2edb440000000p-27f}, {0x1.857f420000000p-1f, -0x1.0c149c0000000p-26f},
    {0x1.8471a40000000p-1f, 0x1.88f1ec0000000p-27f}, {0x1.8364c20000000p-1f, -0x1.46be080000000p-29f},
    {0x1.82589a0000000p-1f, -0x1.accc7c0000000p-27f}, {0x1.814d2a0000000p-1f, 0x1.ba20dc0000000p-26f},
    {0x1.8042760000000p-1f, -0x1.783cbe0000000p-26f}, {0x1.7f38780000000p-1f, 0x1.2471240000000p-27f},
    {0x1.7e2f340000000p-1f, -0x1.2616340000000p-26f}, {0x1.7d26a60000000p-1f, 0x1.7fc3780000000p-28f},
    {0x1.7c1ed00000000p-1f, 0x1.30c1320000000p-29f}, {0x1.7b17b00000000p-1f, 0x1.2ed9fc0000000p-26f},
    {0x1.7a11480000000p-1f, -0x1.829fd00000000p-26f}, {0x1.790b940000000p-1f, -0x1.d4f8c20000000p-27f},
    {0x1.7806940000000p-1f, 0x1.fbcba80000000p-26f}, {0x1.77024c0000000p-1f, -0x1.ca923e0000000p-26f},
    {0x1.75feb60000000p-1f, -0x1.37b3060000000p-26f}, {0x1.74fbd40000000p-1f, -0x1.4506800000000p-26f},
    {0x1.73f9a40000000p-1f, 0x1.14b02e0000000p-26f}, {0x1.72f8280000000p-1f, 0x1.bab4220000000p-27f},
    {0x1.71f75e0000000p-1f, 0x1.1d8bee0000000p-26f}, {0x1.70f7460000000p-1f, 0x1.bd0ba20000000p-27f},
    {0x1.6ff7e00000000p-1f, -0x1.ab9ae00000000p-27f}, {0x1.6ef92a0000000p-1f, -0x1.e9b1460000000p-27f},
    {0x1.6dfb240000000p-1f, -0x1.cd72e80000000p-28f}, {0x1.6cfdce0000000p-1f, -0x1.15c4de0000000p-28f},
    {0x1.6c01280000000p-1f, -0x1.5e84a80000000p-26f}, {0x1.6b05300000000p-1f, -0x1.62ba300000000p-27f},
    {0x1.6a09e60000000p-1f, 0x1.9fcef40000000p-27f}, {0x1.690f4c0000000p-1f, -0x1.cc2d580000000p-26f},
    {0x1.68155e0000000p-1f, -0x1.766ad20000000p-26f},
};
__device__ const float2 COSH_DF[10] = {
    {0x1.0000000000000p+0f, 0x0.0p+0f}, {0x1.0000000000000p-1f, 0x0.0p+0f},
    {0x1.5555560000000p-5f, -0x1.5555560000000p-30f}, {0x1.6c16c20000000p-10f, -0x1.27d27e0000000p-35f},
    {0x1.a01a020000000p-16f, -0x1.7f97fa0000000p-42f}, {0x1.27e4fc0000000p-22f, -0x1.10ec140000000p-47f},
    {0x1.1eed8e0000000p-29f, 0x1.ff1b120000000p-54f}, {0x1.93974a0000000p-37f, 0x1.180f940000000p-62f},
    {0x1.ae7f3e0000000p-45f, 0x1.ccee080000000p-71f}, {0x1.6827860000000p-53f, 0x1.dcbecc0000000p-80f},
};
__device__ const float2 SINH_DF[9] = {
    {0x1.0000000000000p+0f, 0x0.0p+0f}, {0x1.5555560000000p-3f, -0x1.5555560000000p-28f},
    {0x1.1111120000000p-7f, -0x1.ddddde0000000p-32f}, {0x1.a01a020000000p-13f, -0x1.7f97fa0000000p-39f},
    {0x1.71de3a0000000p-19f, 0x1.55b1cc0000000p-45f}, {0x1.ae64560000000p-26f, 0x1.fd51380000000p-52f},
    {0x1.6124620000000p-33f, -0x1.8af25e0000000p-58f}, {0x1.ae7f3e0000000p-41f, 0x1.ccee080000000p-67f},
    {0x1.952c780000000p-49f, -0x1.f9ea560000000p-74f},
};
constexpr float DF_LN2_256_1 = 0x1.6300000000000p-9f;
constexpr float DF_LN2_256_2 = -0x1.bd00000000000p-21f;
constexpr float DF_LN2_256_3 = -0x1.05c6100000000p-37f;
constexpr float DF_INV_LN2_256 = 0x1.7154760000000p+8f;
constexpr float DF_PIO2_1 = 0x1.9220000000000p+0f;
constexpr float DF_PIO2_2 = -0x1.2ae0000000000p-18f;
constexpr float DF_PIO2_3 = -0x1.de973e0000000p-31f;
constexpr float DF_PIO2_4 = 0x1.a626340000000p-58f;
constexpr float DF_TWO_OVER_PI = 0x1.45f3060000000p-1f;


// ------------------------------------------------------------- arithmetic

struct DF { float hi, lo; };

// Error-free transformations; the __f*_rn intrinsics keep the compiler from
// contracting or reassociating them.
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF dfc(float a) { return {a, 0.0f}; }
__device__ __forceinline__ DF dfc(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ DF dneg(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF dadd(DF x, DF y) {
    DF s = two_sum(x.hi, y.hi);
    const DF t = two_sum(x.lo, y.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ DF dsub(DF x, DF y) { return dadd(x, dneg(y)); }
// Cheaper sums where the operands cannot cancel. dadd_q: |x| >= |y| (or
// x == 0); dadd_s: any operands, error bounded by the sum of their
// magnitudes (so only for sums without cancellation).
__device__ __forceinline__ DF dadd_q(DF x, DF y) {
    const DF s = fast_two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF dadd_s(DF x, DF y) {
    const DF s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF dadd_f(DF x, float y) {
    const DF s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ DF dmul(DF x, DF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ DF dmul_f(DF x, float y) {
    const float p = __fmul_rn(x.hi, y);
    float e = __fmaf_rn(x.hi, y, -p);
    e = __fmaf_rn(x.lo, y, e);
    return fast_two_sum(p, e);
}
// x * 2^k for a power of two p2 (exact unless the result leaves the range)
__device__ __forceinline__ DF dscale(DF x, float p2) { return {__fmul_rn(x.hi, p2), __fmul_rn(x.lo, p2)}; }

// A double as hi + lo (hi its nearest float, lo the nearest float of the
// rest): the values of the FP64 records, k and the test velocity.
__host__ __device__ __forceinline__ void split_double(double v, float* hi, float* lo) {
    const float h = (float)v;
    *hi = h;
    *lo = (float)(v - (double)h);
}
__device__ __forceinline__ DF from_double(double v) {
    DF r;
    split_double(v, &r.hi, &r.lo);
    return r;
}
// float -> double on the integer pipe, exactly, for normal floats and zero;
// a subnormal float (only the low word of a value near the bottom of the
// float range) flushes to a signed zero.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long bits = sign | ((unsigned long long)(e + (1023u - 127u)) << 52) |
                                    ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)(e == 0u ? sign : bits));
}
__device__ __forceinline__ double to_double(DF x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

// ------------------------------------------------------------- functions

// e^r - 1 for |r| <= ln2/512 (+ rounding): r + r^2/2 in double-float, then
// r^3/6 + r^4/24 in float (below 2^-48 of the sum's error budget; the next
// term is < 4e-17).
__device__ __forceinline__ DF dexpm1_small(DF r) {
    const DF r2 = dscale(dmul(r, r), 0.5f);
    const float rh = r.hi;
    const float t = __fmul_rn(__fmul_rn(__fmul_rn(rh, rh), rh),
                              __fmaf_rn(rh, 1.0f / 24.0f, 1.0f / 6.0f));
    return dadd_q(dadd_q(r, r2), dfc(t));
}

// y - n ln2/256 for y <= 0 and n = rint(y 256/ln2): y.hi - n L1 is exact
// (Sterbenz), n L2 is exact, n L3 enters as an exact product.
__device__ __forceinline__ DF dreduce(DF y, float nf) {
    const float a = __fsub_rn(y.hi, __fmul_rn(nf, DF_LN2_256_1));
    DF r = two_sum(a, y.lo);
    r = dadd_f(r, -__fmul_rn(nf, DF_LN2_256_2));
    return dsub(r, two_prod(nf, DF_LN2_256_3));
}

// e^-x for x >= 0 (0 once e^-x is below the float range: such terms are
// scaled exponentials next to O(1) ones).
__device__ __forceinline__ DF dexp_neg(DF x) {
    if (!(x.hi < 87.0f)) return {0.0f, 0.0f};
    const DF y = dneg(x);
    const float nf = rintf(__fmul_rn(y.hi, DF_INV_LN2_256));  // -32k <= n <= 0
    const DF em1 = dexpm1_small(dreduce(y, nf));
    const int n = (int)nf;
    const int j = n & 255;
    const int m = n >> 8;  // arithmetic shift: n = 256 m + j
    const DF t = dfc(EXP2_DF[j]);
    const DF v = dadd_q(t, dmul(t, em1));  // 2^(j/256) e^r, in [1, 2)
    return dscale(v, __int_as_float((m + 127) << 23));
}

// e^y - 1 for y <= 0. Kept out of line (called three times per element):
// the element's code must stay within the instruction cache.
static __device__ __noinline__ DF dexpm1_neg(DF y) {
    if (y.hi > -0.35f) {
        const float nf = rintf(__fmul_rn(y.hi, DF_INV_LN2_256));  // -130 <= n <= 0
        const int i = -(int)nf;
        const DF em1 = dexpm1_small(dreduce(y, nf));
        // |2^(-i/256) - 1| >= 2.7e-3 > |2^(-i/256)(e^r - 1)| for i >= 1
        return dadd_q(dfc(EXPM1_DF[i]), dmul(dfc(EXP2N_DF[i]), em1));
    }
    return dadd_q(dfc(-1.0f), dexp_neg(dneg(y)));
}

// 1/sqrt(x), x > 0: the SFU estimate, one float Newton step, one
// double-float Newton step.
__device__ __forceinline__ DF drsqrt(DF x) {
    float y = rsqrtf(x.hi);
    y = __fmul_rn(y, __fmaf_rn(-0.5f * x.hi, __fmul_rn(y, y), 1.5f));
    const DF e = dadd_f(dneg(dmul(x, two_prod(y, y))), 1.0f);  // 1 - x y^2
    return dadd_q(dfc(y), dmul_f(e, 0.5f * y));
}

// 1/x, x != 0.
__device__ __forceinline__ DF drcp(DF x) {
    const float y = __frcp_rn(x.hi);
    const DF e = dadd_f(dneg(dmul_f(x, y)), 1.0f);  // 1 - x y
    return dadd_q(dfc(y), dmul_f(e, y));
}

// cosh(x) - 1 and sinh(x)/x from u = x^2 (either sign: cos - 1, sin/x for
// u < 0), |u| < 1: cosh x - 1 = u sum_{n>=1} u^(n-1)/(2n)!. Terms from
// u^5/12! (of the cosh sum) and u^5/11! (sinh/x) up are summed in float:
// each is below 2^-24 * 2^-24 of its sum.
__device__ __forceinline__ void dseries(DF u, DF* chm1, DF* sh) {
    const float uf = u.hi;
    float c = __fmaf_rn(uf, COSH_DF[9].x, COSH_DF[8].x);
    c = __fmaf_rn(c, uf, COSH_DF[7].x);
    c = __fmaf_rn(c, uf, COSH_DF[6].x);
    float s = __fmaf_rn(uf, SINH_DF[8].x, SINH_DF[7].x);
    s = __fmaf_rn(s, uf, SINH_DF[6].x);
    s = __fmaf_rn(s, uf, SINH_DF[5].x);
    DF pc = dfc(c), ps = dfc(s);
#pragma unroll
    for (int n = 5; n >= 1; --n) pc = dadd_q(dfc(COSH_DF[n]), dmul(pc, u));  // |u| < 1
#pragma unroll
    for (int n = 4; n >= 0; --n) ps = dadd_q(dfc(SINH_DF[n]), dmul(ps, u));
    *chm1 = dmul(u, pc);
    *sh = ps;
}

// sin x and cos x for x >= 0 in double-float. Cody-Waite reduction by the
// nearest multiple j of pi/2, r = x - j (P1 + P2 + P3 + P4): j P1 and j P2
// are exact floats for j < 2^12, j P3 an exact product pair, j P4 a rounded
// float, and the four parts sum to pi/2 within 2^-80, so each step of the
// reduction adds an error of about 2^-47 |r| and the constant none that
// matters. Then cos r - 1 and sin r / r from dseries in u = -r^2
// (|u| <= 0.62), and the quadrant j mod 4. Larger arguments (j >= 2^12,
// x above 6433) take FP64's sincos, split.
__device__ __forceinline__ void dsincos(DF x, DF* sn, DF* cs) {
    const float jf = rintf(__fmul_rn(x.hi, DF_TWO_OVER_PI));
    if (!(jf < 4096.0f)) {
        double s, c;
        sincos(to_double(x), &s, &c);
        *sn = from_double(s);
        *cs = from_double(c);
        return;
    }
    DF r = dadd_f(two_sum(x.hi, -__fmul_rn(jf, DF_PIO2_1)), x.lo);
    r = dadd_f(r, -__fmul_rn(jf, DF_PIO2_2));
    r = dsub(r, two_prod(jf, DF_PIO2_3));
    r = dadd_f(r, -__fmul_rn(jf, DF_PIO2_4));
    DF cm1, sx;
    dseries(dneg(dmul(r, r)), &cm1, &sx);
    const DF s_r = dmul(r, sx);
    const DF c_r = dadd_q(dfc(1.0f), cm1);
    const int q = ((int)jf) & 3;
    const DF a = (q & 1) ? c_r : s_r;
    const DF c = (q & 1) ? s_r : c_r;
    *sn = (q & 2) ? dneg(a) : a;
    *cs = ((q + 1) & 2) ? dneg(c) : c;
}

// U1 = C - 1 (cosh - 1 unscaled) in the series branch, where E = 1.
struct WaveDF { DF E, C, Sd, Sm, U1; bool series; };

// The scaled even functions of masw_device.cuh::wave_fns in double-float
// (out of line: called twice per element). DDTRIG: the trigonometric branch
// (k h |w| >= 1, w imaginary) in double-float too (dsincos); otherwise FP64's
// sincos, split.
template <bool DDTRIG>
static __device__ __noinline__ WaveDF wave_df(DF kh, DF kh2, DF w2) {
    const DF u = dmul(kh2, w2);
    WaveDF o;
    o.series = fabsf(u.hi) < (float)SERIES_U;
    o.U1 = dfc(0.0f);
    if (o.series) {
        DF ps;
        dseries(u, &o.U1, &ps);
        const DF khps = dmul(kh, ps);
        o.E = dfc(1.0f);
        o.C = dadd_q(dfc(1.0f), o.U1);
        o.Sd = khps;
        o.Sm = dmul(w2, khps);
    } else if (w2.hi > 0.0f) {
        const DF rw = drsqrt(w2);
        const DF w = dmul(w2, rw);
        const DF E = dexp_neg(dmul(kh, w));
        const DF E2 = dmul(E, E);
        const DF t = dscale(dadd_q(dfc(1.0f), dneg(E2)), 0.5f);
        o.E = E;
        o.C = dscale(dadd_q(dfc(1.0f), E2), 0.5f);
        o.Sd = dmul(t, rw);
        o.Sm = dmul(t, w);
    } else if (DDTRIG) {  // k h |w| >= 1 with w imaginary
        const DF nw2 = dneg(w2);
        const DF rw = drsqrt(nw2);
        const DF w = dmul(nw2, rw);
        DF sn, cs;
        dsincos(dmul(kh, w), &sn, &cs);
        o.E = dfc(1.0f);
        o.C = cs;
        o.Sd = dmul(sn, rw);
        o.Sm = dneg(dmul(w, sn));
    } else {  // k h |w| >= 1 with w imaginary: FP64 sincos, split
        const double nw2 = -to_double(w2);
        const double rw = rsqrt(nw2);
        const double w = nw2 * rw;
        double sn, cs;
        sincos(to_double(kh) * w, &sn, &cs);
        o.E = dfc(1.0f);
        o.C = from_double(cs);
        o.Sd = from_double(sn * rw);
        o.Sm = from_double(-w * sn);
    }
    return o;
}

// Double-float layer record, from the FP64 record's values: (hi, lo) of h,
// 1/alpha^2, 1/beta^2, 1/beta^2 - 1/alpha^2, 1/rho, beta^2 (12 floats).
constexpr int LAYER_STRIDE_DF = 12;
__host__ __device__ __forceinline__ void df_record(const double* L, float* out) {
    const double v[6] = {L[L_H], L[L_IA2], L[L_IB2], L[L_IB2] - L[L_IA2], L[L_IRHO],
                         L[L_BETA] * L[L_BETA]};
    for (int i = 0; i < 6; ++i) split_double(v[i], out + 2 * i, out + 2 * i + 1);
}

// The element's denominator and six numerators as double-floats (the
// values of LayerNum).
struct LayerNumDD { DF Dh, n00, n01, n11, ce, cf, cg; };

// The element's denominator and numerators before the 1/(rho c^2) and
// beta^2/c^2 factors of layer_numerators_dd.
struct ElemDD { DF Dh, A1, D1, B1, E1, F1, G1; };

// The plain forms of masw_device.cuh::layer_numerators in double-float, for
// a layer whose shear wave is not evanescent (c >= beta_i). Out of line: few
// layers of a certificate take it, and the hot branch of the element, below
// the shear speed, then stays compact in the instruction cache.
template <bool DDTRIG>
static __device__ __noinline__ ElemDD plain_numerators_dd(DF kh, DF r2, DF s2) {
    const DF kh2 = dmul(kh, kh);
    const WaveDF Rw = wave_df<DDTRIG>(kh, kh2, r2);
    const WaveDF Sw = wave_df<DDTRIG>(kh, kh2, s2);
    // both in the series (thin layer): E = 1 and C = 1 + U1, so
    // E_r E_s - C_r C_s = -(U1_r + U1_s + U1_r U1_s) and C_s - C_r =
    // U1_s - U1_r, without the cancellation of differences of numbers
    // near 1 (those would lose digits as 1 / (k h)^2)
    const bool ser = Rw.series && Sw.series;
    const DF u = ser ? dneg(dadd(dadd(Rw.U1, Sw.U1), dmul(Rw.U1, Sw.U1)))
                     : dsub(dmul(Rw.E, Sw.E), dmul(Rw.C, Sw.C));
    const DF SdSd = dmul(Rw.Sd, Sw.Sd);
    ElemDD e;
    e.Dh = dadd(dscale(u, 2.0f), dadd(dmul(Rw.Sm, Sw.Sm), SdSd));
    e.A1 = dsub(dmul(Rw.C, Sw.Sd), dmul(Sw.C, Rw.Sm));
    e.D1 = dsub(dmul(Sw.C, Rw.Sd), dmul(Rw.C, Sw.Sm));
    e.B1 = dneg(dadd(dmul(dadd_f(s2, 3.0f), u),
                     dadd(dmul(Sw.Sm, dadd(dscale(Rw.Sm, 2.0f), Rw.Sd)), SdSd)));
    e.E1 = dsub(dmul(Rw.Sm, Sw.E), dmul(Rw.E, Sw.Sd));
    e.F1 = ser ? dsub(Sw.U1, Rw.U1) : dsub(dmul(Rw.E, Sw.C), dmul(Rw.C, Sw.E));
    e.G1 = dsub(dmul(Sw.Sm, Rw.E), dmul(Sw.E, Rw.Sd));
    return e;
}

// layer_numerators (masw_device.cuh) in double-float: the same quantities as
// LayerNum, kept as double-floats. R = the record (12 floats); k, c^2 and
// 1/c^2 as double-floats. DDTRIG as for wave_df (the leaky continuation,
// where most layers are above their shear speed).
template <bool DDTRIG = false>
__device__ __forceinline__ LayerNumDD layer_numerators_dd(const float* __restrict__ R, DF k, DF c2,
                                                          DF ic2) {
    const float4 A = *reinterpret_cast<const float4*>(R);
    const float4 B = *reinterpret_cast<const float4*>(R + 4);
    const float4 Cc = *reinterpret_cast<const float4*>(R + 8);
    const DF h = {A.x, A.y}, ia2 = {A.z, A.w}, ib2 = {B.x, B.y}, dib = {B.z, B.w};
    const DF irho = {Cc.x, Cc.y}, b2 = {Cc.z, Cc.w};
    const DF one = dfc(1.0f);
    const DF kh = dmul(k, h);
    const DF q = dmul(c2, ib2);
    const DF pp = dmul(c2, ia2);
    const DF r2 = dsub(one, pp);
    const DF s2 = dsub(one, q);
    DF Dh, A1, D1, B1, E1, F1, G1;
    if (s2.hi > 0.0f) {
        // r, s real: every term scaled by exp(-x_r - x_s), no cancellation
        const DF rwr = drsqrt(r2), rws = drsqrt(s2);
        const DF r = dmul(r2, rwr), s = dmul(s2, rws);
        const DF emr1 = dexpm1_neg(dneg(dmul(kh, r)));  // exp(-x_r) - 1
        const DF ems1 = dexpm1_neg(dneg(dmul(kh, s)));
        const DF Er = dadd_q(one, emr1), Es = dadd_q(one, ems1);      // in (0, 1]
        const DF hr = dscale(dmul(emr1, dadd_q(one, Er)), -0.5f);  // exp(-x) sinh x
        const DF hs = dscale(dmul(ems1, dadd_q(one, Es)), -0.5f);
        const DF cr = dadd_q(one, dneg(hr)), cs = dadd_q(one, dneg(hs));  // exp(-x) cosh x
        const DF rs = dmul(r, s);
        const DF irs = drcp(dadd_s(r, s));
        // E_s - E_r = -E_s (exp(-(x_r - x_s)) - 1), x_r - x_s = k h c^2 (1/b^2 - 1/a^2)/(r + s)
        const DF dE = dneg(dmul(Es, dexpm1_neg(dneg(dmul(dmul(kh, dmul(c2, dib)), irs)))));
        // 1 - E_r E_s = -(e_r + e_s + e_r e_s), e = exp(-x) - 1 <= 0: no cancellation
        const DF omP = dneg(dadd_s(dadd_s(emr1, ems1), dmul(emr1, ems1)));
        const DF om = dmul(dadd_s(dadd_s(pp, q), dneg(dmul(pp, q))), drcp(dadd_q(one, rs)));  // 1 - rs
        const DF shd = dscale(dmul(dE, dadd_s(Es, Er)), 0.5f);  // exp(-x_r-x_s) sinh(x_r-x_s)
        const DF sdr = dmul(hr, rwr), sds = dmul(hs, rws);
        Dh = dsub(dmul(dmul(dmul(om, om), sdr), sds), dmul(dE, dE));
        A1 = dmul(dsub(dmul(dmul(om, cs), hr), shd), rws);
        D1 = dmul(dadd_s(dmul(dmul(om, cr), hs), shd), rwr);
        const DF K2 = dadd_s(dmul(dadd_q(dfc(4.0f), dneg(q)), rs),
                             dadd_s(dscale(dmul(rs, rs), 2.0f), dadd_q(one, s2)));
        B1 = dscale(dmul(dadd(dmul(dmul(omP, omP), dmul(om, dsub(q, dscale(om, 2.0f)))),
                              dmul(dmul(dE, dE), K2)),
                         dmul(rwr, rws)),
                    0.25f);
        F1 = dscale(dmul(dE, omP), -0.5f);
        const DF dS = dscale(dmul(dE, dadd_q(one, dmul(Er, Es))), 0.5f);
        E1 = dmul(dsub(dS, dmul(om, dmul(Es, hr))), rws);
        G1 = dneg(dmul(dadd_s(dmul(om, dmul(Er, hs)), dS), rwr));
    } else {
        const ElemDD e = plain_numerators_dd<DDTRIG>(kh, r2, s2);
        Dh = e.Dh;
        A1 = e.A1;
        D1 = e.D1;
        B1 = e.B1;
        E1 = e.E1;
        F1 = e.F1;
        G1 = e.G1;
    }
    const DF irc2 = dmul(irho, ic2);  // 1 / (rho c^2)
    return LayerNumDD{dmul(Dh, irc2), A1, dmul(dmul(b2, ic2), B1), D1, E1, F1, G1};
}

// layer_numerators_dd rounded to doubles (the element check compares them
// with the FP64 element).
__device__ __forceinline__ LayerNum layer_numerators_df(const float* __restrict__ R, DF k, DF c2,
                                                        DF ic2) {
    const LayerNumDD d = layer_numerators_dd(R, k, c2, ic2);
    return LayerNum{to_double(d.Dh), to_double(d.n00), to_double(d.n01), to_double(d.n11),
                    to_double(d.ce), to_double(d.cf), to_double(d.cg)};
}

// ------------------------------------------------ Schur step in double-float
//
// GB300 issues 2 FP64 operations per clock per SM against 128 FP32 ones.
// With the element on the FP32 pipe the FP64 Schur step (29 FP64 operations a
// layer, plus the 7 conversions of the element's values) set the pace of the
// certificate, so the step runs in double-float too: the homogeneous
// division-free recurrence of schur_layer, each FP64 product a dmul and each
// FP64 fused multiply-add a dfma, the state renormalised by a power of two per
// layer (exponent on the integer pipe). Relative rounding of about 2^-47 per
// operation, against the element's own error of about 1e-13 relative.

// a * b + c for any signs (cancellation included): the product's rounding
// error and cross terms are carried into the low word, the leading words are
// summed error-free (two_sum). Error about 2^-47 (|a b| + |c|). The last
// renormalisation is a fast_two_sum: where the leading sum cancelled so far
// that the low word t exceeds it, that step's error stays below 2^-23 |t|,
// about 2^-46 (|a b| + |c|), the order of the bound, and the leading word
// keeps the sign of the rounded sum.
__device__ __forceinline__ DF dfma(DF a, DF b, DF c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const DF s = two_sum(p, c.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

struct HStateDD { DF p00, p01, p11, w; };

// exponent field of a float (0: zero or subnormal, 255: inf or NaN)
__device__ __forceinline__ int fexp(float x) { return (__float_as_int(x) >> 23) & 0xff; }

// schur_layer (masw_device.cuh) in double-float: eliminates one layer's top
// node, returns det(Shat) and its first diagonal entry in *s00o. *ok is false
// when the new scale w is zero, subnormal, non-finite or outside
// [2^-125, 2^127), or a new state entry is not finite.
__device__ __forceinline__ DF schur_layer_dd(HStateDD& st, const LayerNumDD& n, bool* ok,
                                             DF* s00o) {
    const DF w = st.w;
    const DF s00 = dfma(n.Dh, st.p00, dmul(w, n.n00));
    const DF s01 = dfma(n.Dh, st.p01, dmul(w, n.n01));
    const DF s11 = dfma(n.Dh, st.p11, dmul(w, n.n11));
    const DF det = dfma(s00, s11, dneg(dmul(s01, s01)));
    // T = adj(Shat) * [[ce, cf], [-cf, cg]];  Q = [[ce, -cf], [cf, cg]] * T
    const DF t00 = dfma(s11, n.ce, dmul(s01, n.cf));
    const DF t01 = dfma(s11, n.cf, dneg(dmul(s01, n.cg)));
    const DF t10 = dneg(dfma(s01, n.ce, dmul(s00, n.cf)));
    const DF t11 = dfma(s00, n.cg, dneg(dmul(s01, n.cf)));
    const DF q00 = dfma(n.ce, t00, dneg(dmul(n.cf, t10)));
    const DF q01 = dfma(n.ce, t01, dneg(dmul(n.cf, t11)));
    const DF q11 = dfma(n.cf, t01, dmul(n.cg, t11));
    const DF p00 = dfma(n.n00, det, dneg(dmul(w, q00)));
    const DF p01 = dfma(dneg(n.n01), det, dneg(dmul(w, q01)));
    const DF p11 = dfma(n.n11, det, dneg(dmul(w, q11)));
    const DF wn = dmul(n.Dh, det);
    // scale by 2^(127 - e), e = the exponent field of wn: w to [1, 2)
    const int ew = fexp(wn.hi);
    const float sc = __int_as_float((254 - min(max(ew, 2), 253)) << 23);
    st.p00 = dscale(p00, sc);
    st.p01 = dscale(p01, sc);
    st.p11 = dscale(p11, sc);
    st.w = dscale(wn, sc);
    *ok = ew >= 2 && ew <= 253 && fexp(st.p00.hi) != 255 && fexp(st.p01.hi) != 255 &&
          fexp(st.p11.hi) != 255;
    *s00o = s00;
    return det;
}

// Number of negative eigenvalues of K(k, c) from the FP64 recurrence over the
// finite layers' elements in double-float (Sylvester's law of inertia over the
// 2x2 Schur pivots S_j = Shat_j / (w Dh): a pivot with det < 0 has one, one
// with det > 0 has two when its diagonal is negative; a zero determinant
// counts as one; -1 when the rescaling failed). Its parity is the sign of
// det K. DD: the Schur step in double-float too (schur_layer_dd), for points
// inside the pole-free range only: no element is near a pole there, while
// above it the recurrence's cancellation next to the poles magnifies the
// step's rounding (with it the higher-mode search missed 3 of 1.7 M events
// that the FP64 scan finds); otherwise the FP64 step (schur_layer). laydf:
// the N finite layers' double-float records, or nullptr to split the FP64
// records on the fly (the same values). Requires c < beta_halfspace.
template <bool DD>
__device__ __forceinline__ int det_inertia_t(const float* __restrict__ laydf,
                                             const double* __restrict__ lay, int N, double k,
                                             double c) {
    const double c2 = c * c;
    const DF kd = from_double(k), cd = from_double(c);
    const DF c2d = dmul(cd, cd);
    const DF ic2d = drcp(c2d);
    HStateDD sd{dfc(0.0f), dfc(0.0f), dfc(0.0f), dfc(1.0f)};
    HState st{0.0, 0.0, 0.0, 1.0};
    int cnt = 0;
    for (int j = 0; j < N; ++j) {
        float rec[LAYER_STRIDE_DF];
        const float* R = laydf ? laydf + j * LAYER_STRIDE_DF : rec;
        if (!laydf) df_record(lay + j * LAYER_STRIDE, rec);
        const LayerNumDD nd = layer_numerators_dd(R, kd, c2d, ic2d);
        bool ok;
        if (DD) {
            const bool f_neg = (sd.w.hi < 0.0f) != (nd.Dh.hi < 0.0f);  // sign of w Dh
            DF s00;
            const DF det = schur_layer_dd(sd, nd, &ok, &s00);
            cnt += det.hi < 0.0f ? 1
                                 : (det.hi > 0.0f ? (((s00.hi < 0.0f) != f_neg) ? 2 : 0) : 1);
        } else {
            const LayerNum n{to_double(nd.Dh), to_double(nd.n00), to_double(nd.n01),
                             to_double(nd.n11), to_double(nd.ce), to_double(nd.cf),
                             to_double(nd.cg)};
            const bool f_neg = wprod_lt0(st.w, n.Dh);
            double sv[3];
            const double det = schur_layer(st, n, &ok, sv);
            cnt += lt0(det) ? 1 : (gt0(det) ? ((lt0(sv[0]) != f_neg) ? 2 : 0) : 1);
        }
        if (!ok) return -1;
    }
    if (DD) st = HState{to_double(sd.p00), to_double(sd.p01), to_double(sd.p11), to_double(sd.w)};
    HalfNum hn = halfspace_numerators(lay + N * LAYER_STRIDE, c2);
    const bool f_neg = wprod_lt0(st.w, hn.den);
    double s00 = fma(hn.den, st.p00, st.w * hn.m00);
    double s01 = fma(hn.den, st.p01, st.w * hn.m01);
    double s11 = fma(hn.den, st.p11, st.w * hn.m11);
    double det = fma(s00, s11, -s01 * s01);
    cnt += lt0(det) ? 1 : (gt0(det) ? ((lt0(s00) != f_neg) ? 2 : 0) : 1);
    return cnt;
}

// Out of line: each is called from several places, and one copy of the
// element keeps a kernel within the instruction cache.
static __device__ __noinline__ int det_inertia_df(const float* __restrict__ laydf,
                                                  const double* __restrict__ lay, int N, double k,
                                                  double c) {
    return det_inertia_t<false>(laydf, lay, N, k, c);
}
static __device__ __noinline__ int det_inertia_dd(const float* __restrict__ laydf,
                                                  const double* __restrict__ lay, int N, double k,
                                                  double c) {
    return det_inertia_t<true>(laydf, lay, N, k, c);
}

// Sign of Re det K(k, c) for any c > 0 (masw_device.cuh::det_sign_leaky)
// with each finite layer's element in double-float, trigonometric branch
// included (layer_numerators_dd<true>): above the half-space shear speed
// most layers are above their own, and FP64's sincos there set the pace of
// the FP64 form. FP64STEP false: the Schur step in double-float too
// (schur_layer_dd), so the FP64 pipe carries only the complex half-space
// pivot (leaky_halfspace_sign); true: the Schur step in FP64 (schur_layer).
// Far above the pole-free range the recurrence cancels next to the poles and
// the double-float step's sign can differ from the FP64 step's there: the
// continuation locates with the first and confirms each change with the
// second. 0 for an exact zero or a failed rescaling, as det_sign_leaky.
// laydf: the N finite layers' double-float records.
template <bool FP64STEP>
__device__ __forceinline__ int det_sign_leaky_t(const float* __restrict__ laydf,
                                                const double* __restrict__ lay, int N, double k,
                                                double c) {
    const double c2 = c * c;
    const DF kd = from_double(k), cd = from_double(c);
    const DF c2d = dmul(cd, cd);
    const DF ic2d = drcp(c2d);
    HStateDD sd{dfc(0.0f), dfc(0.0f), dfc(0.0f), dfc(1.0f)};
    HState st{0.0, 0.0, 0.0, 1.0};
    int sg = 1;
    for (int j = 0; j < N; ++j) {
        const LayerNumDD nd = layer_numerators_dd<true>(laydf + j * LAYER_STRIDE_DF, kd, c2d, ic2d);
        bool ok;
        if (FP64STEP) {
            const LayerNum n{to_double(nd.Dh), to_double(nd.n00), to_double(nd.n01),
                             to_double(nd.n11), to_double(nd.ce), to_double(nd.cf),
                             to_double(nd.cg)};
            sg *= sgn(schur_layer(st, n, &ok));
        } else {
            DF s00;
            const DF det = schur_layer_dd(sd, nd, &ok, &s00);
            sg *= det.hi > 0.0f ? 1 : (det.hi < 0.0f ? -1 : 0);
        }
        if (!ok) return 0;
    }
    if (!FP64STEP)
        st = HState{to_double(sd.p00), to_double(sd.p01), to_double(sd.p11), to_double(sd.w)};
    return sg * leaky_halfspace_sign(lay + N * LAYER_STRIDE, c2, st);
}
// Out of line, one for each step: the scan kernel holds one, the check
// kernel the other.
static __device__ __noinline__ int det_sign_leaky_dd(const float* __restrict__ laydf,
                                                     const double* __restrict__ lay, int N,
                                                     double k, double c) {
    return det_sign_leaky_t<false>(laydf, lay, N, k, c);
}
static __device__ __noinline__ int det_sign_leaky_df(const float* __restrict__ laydf,
                                                     const double* __restrict__ lay, int N,
                                                     double k, double c) {
    return det_sign_leaky_t<true>(laydf, lay, N, k, c);
}

// Wittrick-Williams mode count of the layered structure below c, split as
// (s, J0): s = negative eigenvalues of K (det_inertia_df; -1 when the
// rescaling failed), J0 = clamped modes of all finite layers (clamped_modes,
// from the FP64 records; the half-space has none below its shear speed).
// J = J0 + s, the number of modes below c, never decreases with c, and
// neither does T = J + J0 = s + 2 J0, whose parity is that of s: det K changes
// sign between two test velocities exactly when T jumps by an odd amount
// between them. laydf as for det_inertia_df. Requires c < beta_halfspace.
// Out of line: the mode-count searches call it from several places.
static __device__ __noinline__ int mode_count_T_df(const float* __restrict__ laydf,
                                      const double* __restrict__ lay, int N, double k, double c,
                                      int* s_out) {
    const int s = det_inertia_df(laydf, lay, N, k, c);
    const double c2 = c * c;
    int j0 = 0;
    for (int j = 0; j < N; ++j) j0 += clamped_modes(lay + j * LAYER_STRIDE, k, c2);
    *s_out = s;
    return s < 0 ? -1 : s + 2 * j0;
}

}  // namespace masw
