// ksdf_exp.cuh -- binary64 exp(-lambda r^2) for the kernel matrix of the fit, and exact bit-level
// conversions between binary64 and binary32 that keep the scarce FP64 pipe free.
//
// The argument is carried in units of ln2 / 2^16: e = (2^16 / ln2) lambda r^2 >= 0 and the value is
// 2^(-e / 2^16).  With n = round(e) = 2^16 m + 2^8 a + b and r = e - n (|r| <= 1/2):
//   2^(-e / 2^16) = 2^-m * T1[a] * T2[b] * (1 + q),  q = r (C2 r - C1) = exp(-C1 r) - 1 + O(3e-17),
// T1[a] = 2^(-a/256), T2[b] = 2^(-b/65536), C1 = ln2 / 2^16 (a two-level table variant of P. T. P. Tang's
// table-driven exponential, ACM TOMS 15(2), 1989).  n and r are extracted from the bits of e with integer
// operations (r as a 40-bit fixed-point fraction, exact for e < 2^22), so an entry costs 4 FP64 operations
// after its argument; the result is within about 2.5 units of 2^-53 (two table roundings and two
// operation roundings).  Valid for 0 <= e < 2^22 (lambda r^2 < 44).
// Constants from gen_exp_consts.py (60-digit decimal arithmetic).
#pragma once

namespace ksdf {

constexpr double kExpC1 = 0x1.62e42fefa39efp-17;
constexpr double kExpC2 = 0x1.ebfbdff82c58fp-35;
constexpr double kExpQ16PerNat = 0x1.71547652b82fep+16;

__device__ double kExpT1[256] = {  // 2^(-j/256)
    0x1.0000000000000p+0, 0x1.fe9d96b2a23d9p-1, 0x1.fd3c22b8f71f1p-1, 0x1.fbdba3692d514p-1,
    0x1.fa7c1819e90d8p-1, 0x1.f91d802243c89p-1, 0x1.f7bfdad9cbe14p-1, 0x1.f6632798844f8p-1,
    0x1.f50765b6e4540p-1, 0x1.f3ac948dd7274p-1, 0x1.f252b376bba97p-1, 0x1.f0f9c1cb6412ap-1,
    0x1.efa1bee615a27p-1, 0x1.ee4aaa2188510p-1, 0x1.ecf482d8e67f1p-1, 0x1.eb9f4867cca6ep-1,
    0x1.ea4afa2a490dap-1, 0x1.e8f7977cdb740p-1, 0x1.e7a51fbc74c83p-1, 0x1.e653924676d76p-1,
    0x1.e502ee78b3ff6p-1, 0x1.e3b333b16ee12p-1, 0x1.e264614f5a129p-1, 0x1.e11676b197d17p-1,
    0x1.dfc97337b9b5fp-1, 0x1.de7d5641c0658p-1, 0x1.dd321f301b460p-1, 0x1.dbe7cd63a8315p-1,
    0x1.da9e603db3285p-1, 0x1.d955d71ff6075p-1, 0x1.d80e316c98398p-1, 0x1.d6c76e862e6d3p-1,
    0x1.d5818dcfba487p-1, 0x1.d43c8eacaa1d6p-1, 0x1.d2f87080d89f2p-1, 0x1.d1b532b08c968p-1,
    0x1.d072d4a07897cp-1, 0x1.cf3155b5bab74p-1, 0x1.cdf0b555dc3fap-1, 0x1.ccb0f2e6d1675p-1,
    0x1.cb720dcef9069p-1, 0x1.ca3405751c4dbp-1, 0x1.c8f6d9406e7b5p-1, 0x1.c7ba88988c933p-1,
    0x1.c67f12e57d14bp-1, 0x1.c544778fafb22p-1, 0x1.c40ab5fffd07ap-1, 0x1.c2d1cd9fa652cp-1,
    0x1.c199bdd85529cp-1, 0x1.c06286141b33dp-1, 0x1.bf2c25bd71e09p-1, 0x1.bdf69c3f3a207p-1,
    0x1.bcc1e904bc1d2p-1, 0x1.bb8e0b79a6f1fp-1, 0x1.ba5b030a1064ap-1, 0x1.b928cf22749e4p-1,
    0x1.b7f76f2fb5e47p-1, 0x1.b6c6e29f1c52ap-1, 0x1.b59728de5593ap-1, 0x1.b468415b749b1p-1,
    0x1.b33a2b84f15fbp-1, 0x1.b20ce6c9a8952p-1, 0x1.b0e07298db666p-1, 0x1.afb4ce622f2ffp-1,
    0x1.ae89f995ad3adp-1, 0x1.ad5ff3a3c2774p-1, 0x1.ac36bbfd3f37ap-1, 0x1.ab0e521356ebap-1,
    0x1.a9e6b5579fdbfp-1, 0x1.a8bfe53c12e59p-1, 0x1.a799e1330b358p-1, 0x1.a674a8af46052p-1,
    0x1.a5503b23e255dp-1, 0x1.a42c980460ad8p-1, 0x1.a309bec4a2d33p-1, 0x1.a1e7aed8eb8bbp-1,
    0x1.a0c667b5de565p-1, 0x1.9fa5e8d07f29ep-1, 0x1.9e86319e32323p-1, 0x1.9d674194bb8d5p-1,
    0x1.9c49182a3f090p-1, 0x1.9b2bb4d53fe0dp-1, 0x1.9a0f170ca07bap-1, 0x1.98f33e47a22a2p-1,
    0x1.97d829fde4e50p-1, 0x1.96bdd9a7670b3p-1, 0x1.95a44cbc8520fp-1, 0x1.948b82b5f98e5p-1,
    0x1.93737b0cdc5e5p-1, 0x1.925c353aa2fe2p-1, 0x1.9145b0b91ffc6p-1, 0x1.902fed0282c8ap-1,
    0x1.8f1ae99157736p-1, 0x1.8e06a5e0866d9p-1, 0x1.8cf3216b5448cp-1, 0x1.8be05bad61778p-1,
    0x1.8ace5422aa0dbp-1, 0x1.89bd0a478580fp-1, 0x1.88ac7d98a6699p-1, 0x1.879cad931a436p-1,
    0x1.868d99b4492edp-1, 0x1.857f4179f5b21p-1, 0x1.8471a4623c7adp-1, 0x1.8364c1eb941f7p-1,
    0x1.82589994cce13p-1, 0x1.814d2add106d9p-1, 0x1.80427543e1a12p-1, 0x1.7f3878491c491p-1,
    0x1.7e2f336cf4e62p-1, 0x1.7d26a62ff86f0p-1, 0x1.7c1ed0130c132p-1, 0x1.7b17b0976cfdbp-1,
    0x1.7a11473eb0187p-1, 0x1.790b938ac1cf6p-1, 0x1.780694fde5d3fp-1, 0x1.77024b1ab6e09p-1,
    0x1.75feb564267c9p-1, 0x1.74fbd35d7cbfdp-1, 0x1.73f9a48a58174p-1, 0x1.72f8286ead08ap-1,
    0x1.71f75e8ec5f74p-1, 0x1.70f7466f42e87p-1, 0x1.6ff7df9519484p-1, 0x1.6ef9298593ae5p-1,
    0x1.6dfb23c651a2fp-1, 0x1.6cfdcddd47645p-1, 0x1.6c012750bdabfp-1, 0x1.6b052fa75173ep-1,
    0x1.6a09e667f3bcdp-1, 0x1.690f4b19e9538p-1, 0x1.68155d44ca973p-1, 0x1.671c1c70833f6p-1,
    0x1.6623882552225p-1, 0x1.652b9febc8fb7p-1, 0x1.6434634ccc320p-1, 0x1.633dd1d1929fdp-1,
    0x1.6247eb03a5585p-1, 0x1.6152ae6cdf6f4p-1, 0x1.605e1b976dc09p-1, 0x1.5f6a320dceb71p-1,
    0x1.5e76f15ad2148p-1, 0x1.5d84590998b93p-1, 0x1.5c9268a5946b7p-1, 0x1.5ba11fba87a03p-1,
    0x1.5ab07dd485429p-1, 0x1.59c0827ff07ccp-1, 0x1.58d12d497c7fdp-1, 0x1.57e27dbe2c4cfp-1,
    0x1.56f4736b527dap-1, 0x1.56070dde910d2p-1, 0x1.551a4ca5d920fp-1, 0x1.542e2f4f6ad27p-1,
    0x1.5342b569d4f82p-1, 0x1.5257de83f4eefp-1, 0x1.516daa2cf6642p-1, 0x1.508417f4531eep-1,
    0x1.4f9b2769d2ca7p-1, 0x1.4eb2d81d8abffp-1, 0x1.4dcb299fddd0dp-1, 0x1.4ce41b817c114p-1,
    0x1.4bfdad5362a27p-1, 0x1.4b17dea6db7d7p-1, 0x1.4a32af0d7d3dep-1, 0x1.494e1e192aed2p-1,
    0x1.486a2b5c13cd0p-1, 0x1.4786d668b3237p-1, 0x1.46a41ed1d0057p-1, 0x1.45c2042a7d232p-1,
    0x1.44e086061892dp-1, 0x1.43ffa3f84b9d4p-1, 0x1.431f5d950a897p-1, 0x1.423fb2709468ap-1,
    0x1.4160a21f72e2ap-1, 0x1.40822c367a024p-1, 0x1.3fa4504ac801cp-1, 0x1.3ec70df1c5175p-1,
    0x1.3dea64c123422p-1, 0x1.3d0e544ede173p-1, 0x1.3c32dc313a8e5p-1, 0x1.3b57fbfec6cf4p-1,
    0x1.3a7db34e59ff7p-1, 0x1.39a401b7140efp-1, 0x1.38cae6d05d866p-1, 0x1.37f26231e754ap-1,
    0x1.371a7373aa9cbp-1, 0x1.36431a2de883bp-1, 0x1.356c55f929ff1p-1, 0x1.3496266e3fa2dp-1,
    0x1.33c08b26416ffp-1, 0x1.32eb83ba8ea32p-1, 0x1.32170fc4cd831p-1, 0x1.31432edeeb2fdp-1,
    0x1.306fe0a31b715p-1, 0x1.2f9d24abd886bp-1, 0x1.2ecafa93e2f56p-1, 0x1.2df961f641589p-1,
    0x1.2d285a6e4030bp-1, 0x1.2c57e39771b2fp-1, 0x1.2b87fd0dad990p-1, 0x1.2ab8a66d10f13p-1,
    0x1.29e9df51fdee1p-1, 0x1.291ba7591bb70p-1, 0x1.284dfe1f56381p-1, 0x1.2780e341ddf29p-1,
    0x1.26b4565e27cddp-1, 0x1.25e85711ece75p-1, 0x1.251ce4fb2a63fp-1, 0x1.2451ffb82140ap-1,
    0x1.2387a6e756238p-1, 0x1.22bdda27912d1p-1, 0x1.21f49917ddc96p-1, 0x1.212be3578a819p-1,
    0x1.2063b88628cd6p-1, 0x1.1f9c18438ce4dp-1, 0x1.1ed5022fcd91dp-1, 0x1.1e0e75eb44027p-1,
    0x1.1d4873168b9aap-1, 0x1.1c82f95281c6bp-1, 0x1.1bbe084045cd4p-1, 0x1.1af99f8138a1cp-1,
    0x1.1a35beb6fcb75p-1, 0x1.1972658375d2fp-1, 0x1.18af9388c8deap-1, 0x1.17ed48695bbc0p-1,
    0x1.172b83c7d517bp-1, 0x1.166a45471c3c2p-1, 0x1.15a98c8a58e51p-1, 0x1.14e95934f312ep-1,
    0x1.1429aaea92de0p-1, 0x1.136a814f204abp-1, 0x1.12abdc06c31ccp-1, 0x1.11edbab5e2ab6p-1,
    0x1.11301d0125b51p-1, 0x1.1073028d7233ep-1, 0x1.0fb66affed31bp-1, 0x1.0efa55fdfa9c5p-1,
    0x1.0e3ec32d3d1a2p-1, 0x1.0d83b23395decp-1, 0x1.0cc922b7247f7p-1, 0x1.0c0f145e46c85p-1,
    0x1.0b5586cf9890fp-1, 0x1.0a9c79b1f3919p-1, 0x1.09e3ecac6f383p-1, 0x1.092bdf66607e0p-1,
    0x1.0874518759bc8p-1, 0x1.07bd42b72a836p-1, 0x1.0706b29ddf6dep-1, 0x1.0650a0e3c1f89p-1,
    0x1.059b0d3158574p-1, 0x1.04e5f72f654b1p-1, 0x1.04315e86e7f85p-1, 0x1.037d42e11bbccp-1,
    0x1.02c9a3e778061p-1, 0x1.02168143b0281p-1, 0x1.0163da9fb3335p-1, 0x1.00b1afa5abcbfp-1,
};
__device__ double kExpT2[256] = {  // 2^(-j/65536)
    0x1.0000000000000p+0, 0x1.fffe9d1c4b0f3p-1, 0x1.fffd3a398c1bbp-1, 0x1.fffbd757c324dp-1,
    0x1.fffa7476f029dp-1, 0x1.fff91197132a2p-1, 0x1.fff7aeb82c251p-1, 0x1.fff64bda3b19fp-1,
    0x1.fff4e8fd40081p-1, 0x1.fff386213aeedp-1, 0x1.fff223462bcd8p-1, 0x1.fff0c06c12a37p-1,
    0x1.ffef5d92ef700p-1, 0x1.ffedfabac2328p-1, 0x1.ffec97e38aea5p-1, 0x1.ffeb350d4996cp-1,
    0x1.ffe9d237fe372p-1, 0x1.ffe86f63a8cacp-1, 0x1.ffe70c9049510p-1, 0x1.ffe5a9bddfc93p-1,
    0x1.ffe446ec6c32bp-1, 0x1.ffe2e41bee8cdp-1, 0x1.ffe1814c66d6ep-1, 0x1.ffe01e7dd5103p-1,
    0x1.ffdebbb039383p-1, 0x1.ffdd58e3934e1p-1, 0x1.ffdbf617e3515p-1, 0x1.ffda934d29412p-1,
    0x1.ffd93083651cfp-1, 0x1.ffd7cdba96e40p-1, 0x1.ffd66af2be95bp-1, 0x1.ffd5082bdc316p-1,
    0x1.ffd3a565efb65p-1, 0x1.ffd242a0f923ep-1, 0x1.ffd0dfdcf8797p-1, 0x1.ffcf7d19edb64p-1,
    0x1.ffce1a57d8d9cp-1, 0x1.ffccb796b9e33p-1, 0x1.ffcb54d690d1fp-1, 0x1.ffc9f2175da54p-1,
    0x1.ffc88f59205cap-1, 0x1.ffc72c9bd8f74p-1, 0x1.ffc5c9df87748p-1, 0x1.ffc467242bd3cp-1,
    0x1.ffc30469c6145p-1, 0x1.ffc1a1b056358p-1, 0x1.ffc03ef7dc36ap-1, 0x1.ffbedc4058171p-1,
    0x1.ffbd7989c9d63p-1, 0x1.ffbc16d431734p-1, 0x1.ffbab41f8eedap-1, 0x1.ffb9516be244bp-1,
    0x1.ffb7eeb92b77bp-1, 0x1.ffb68c076a860p-1, 0x1.ffb529569f6f0p-1, 0x1.ffb3c6a6ca31fp-1,
    0x1.ffb263f7eace3p-1, 0x1.ffb1014a01432p-1, 0x1.ffaf9e9d0d900p-1, 0x1.ffae3bf10fb43p-1,
    0x1.ffacd94607af1p-1, 0x1.ffab769bf57ffp-1, 0x1.ffaa13f2d9262p-1, 0x1.ffa8b14ab2a0fp-1,
    0x1.ffa74ea381efcp-1, 0x1.ffa5ebfd4711ep-1, 0x1.ffa489580206bp-1, 0x1.ffa326b3b2cd8p-1,
    0x1.ffa1c4105965ap-1, 0x1.ffa0616df5ce7p-1, 0x1.ff9efecc88073p-1, 0x1.ff9d9c2c100f5p-1,
    0x1.ff9c398c8de62p-1, 0x1.ff9ad6ee018aep-1, 0x1.ff9974506afd0p-1, 0x1.ff9811b3ca3bdp-1,
    0x1.ff96af181f46ap-1, 0x1.ff954c7d6a1ccp-1, 0x1.ff93e9e3aabd9p-1, 0x1.ff92874ae1285p-1,
    0x1.ff9124b30d5c8p-1, 0x1.ff8fc21c2f595p-1, 0x1.ff8e5f86471e2p-1, 0x1.ff8cfcf154aa5p-1,
    0x1.ff8b9a5d57fd3p-1, 0x1.ff8a37ca51161p-1, 0x1.ff88d5383ff45p-1, 0x1.ff8772a724973p-1,
    0x1.ff861016fefe2p-1, 0x1.ff84ad87cf287p-1, 0x1.ff834af995156p-1, 0x1.ff81e86c50c46p-1,
    0x1.ff8085e00234bp-1, 0x1.ff7f2354a965cp-1, 0x1.ff7dc0ca4656dp-1, 0x1.ff7c5e40d9073p-1,
    0x1.ff7afbb861765p-1, 0x1.ff799930dfa37p-1, 0x1.ff7836aa538e0p-1, 0x1.ff76d424bd353p-1,
    0x1.ff7571a01c987p-1, 0x1.ff740f1c71b70p-1, 0x1.ff72ac99bc905p-1, 0x1.ff714a17fd23bp-1,
    0x1.ff6fe79733706p-1, 0x1.ff6e85175f75dp-1, 0x1.ff6d229881334p-1, 0x1.ff6bc01a98a82p-1,
    0x1.ff6a5d9da5d3bp-1, 0x1.ff68fb21a8b54p-1, 0x1.ff6798a6a14c4p-1, 0x1.ff66362c8f97fp-1,
    0x1.ff64d3b37397bp-1, 0x1.ff63713b4d4adp-1, 0x1.ff620ec41cb0ap-1, 0x1.ff60ac4de1c88p-1,
    0x1.ff5f49d89c91dp-1, 0x1.ff5de7644d0bdp-1, 0x1.ff5c84f0f335ep-1, 0x1.ff5b227e8f0f5p-1,
    0x1.ff59c00d20978p-1, 0x1.ff585d9ca7cdcp-1, 0x1.ff56fb2d24b17p-1, 0x1.ff5598be9741dp-1,
    0x1.ff543650ff7e4p-1, 0x1.ff52d3e45d661p-1, 0x1.ff517178b0f8bp-1, 0x1.ff500f0dfa355p-1,
    0x1.ff4eaca4391b6p-1, 0x1.ff4d4a3b6daa3p-1, 0x1.ff4be7d397e11p-1, 0x1.ff4a856cb7bf5p-1,
    0x1.ff492306cd446p-1, 0x1.ff47c0a1d86f7p-1, 0x1.ff465e3dd9400p-1, 0x1.ff44fbdacfb54p-1,
    0x1.ff439978bbceap-1, 0x1.ff4237179d8b6p-1, 0x1.ff40d4b774eafp-1, 0x1.ff3f725841ec9p-1,
    0x1.ff3e0ffa048fap-1, 0x1.ff3cad9cbcd37p-1, 0x1.ff3b4b406ab75p-1, 0x1.ff39e8e50e3abp-1,
    0x1.ff38868aa75ccp-1, 0x1.ff372431361cfp-1, 0x1.ff35c1d8ba7a9p-1, 0x1.ff345f8134750p-1,
    0x1.ff32fd2aa40b8p-1, 0x1.ff319ad5093d7p-1, 0x1.ff303880640a2p-1, 0x1.ff2ed62cb4710p-1,
    0x1.ff2d73d9fa714p-1, 0x1.ff2c1188360a5p-1, 0x1.ff2aaf37673b7p-1, 0x1.ff294ce78e041p-1,
    0x1.ff27ea98aa638p-1, 0x1.ff26884abc590p-1, 0x1.ff2525fdc3e3fp-1, 0x1.ff23c3b1c103cp-1,
    0x1.ff226166b3b7ap-1, 0x1.ff20ff1c9bfefp-1, 0x1.ff1f9cd379d92p-1, 0x1.ff1e3a8b4d456p-1,
    0x1.ff1cd84416432p-1, 0x1.ff1b75fdd4d1ap-1, 0x1.ff1a13b888f05p-1, 0x1.ff18b174329e7p-1,
    0x1.ff174f30d1db6p-1, 0x1.ff15ecee66a68p-1, 0x1.ff148aacf0ff1p-1, 0x1.ff13286c70e47p-1,
    0x1.ff11c62ce655fp-1, 0x1.ff1063ee5152fp-1, 0x1.ff0f01b0b1dacp-1, 0x1.ff0d9f7407eccp-1,
    0x1.ff0c3d3853883p-1, 0x1.ff0adafd94ac7p-1, 0x1.ff0978c3cb58ep-1, 0x1.ff08168af78cdp-1,
    0x1.ff06b45319479p-1, 0x1.ff05521c30888p-1, 0x1.ff03efe63d4eep-1, 0x1.ff028db13f9a2p-1,
    0x1.ff012b7d37699p-1, 0x1.feffc94a24bc8p-1, 0x1.fefe671807924p-1, 0x1.fefd04e6dfea3p-1,
    0x1.fefba2b6adc3ap-1, 0x1.fefa4087711dep-1, 0x1.fef8de5929f86p-1, 0x1.fef77c2bd8526p-1,
    0x1.fef619ff7c2b3p-1, 0x1.fef4b7d415823p-1, 0x1.fef355a9a456cp-1, 0x1.fef1f38028a82p-1,
    0x1.fef09157a275bp-1, 0x1.feef2f3011bedp-1, 0x1.feedcd097682dp-1, 0x1.feec6ae3d0c10p-1,
    0x1.feeb08bf2078bp-1, 0x1.fee9a69b65a94p-1, 0x1.fee84478a0520p-1, 0x1.fee6e256d0725p-1,
    0x1.fee58035f6099p-1, 0x1.fee41e161116fp-1, 0x1.fee2bbf72199ep-1, 0x1.fee159d92791bp-1,
    0x1.fedff7bc22fdcp-1, 0x1.fede95a013dd6p-1, 0x1.fedd3384fa2fdp-1, 0x1.fedbd16ad5f49p-1,
    0x1.feda6f51a72adp-1, 0x1.fed90d396dd1fp-1, 0x1.fed7ab2229e95p-1, 0x1.fed6490bdb704p-1,
    0x1.fed4e6f682662p-1, 0x1.fed384e21eca3p-1, 0x1.fed222ceb09bep-1, 0x1.fed0c0bc37da7p-1,
    0x1.fecf5eaab4853p-1, 0x1.fecdfc9a269bap-1, 0x1.fecc9a8a8e1cep-1, 0x1.fecb387beb087p-1,
    0x1.fec9d66e3d5d9p-1, 0x1.fec87461851b9p-1, 0x1.fec71255c241ep-1, 0x1.fec5b04af4cfcp-1,
    0x1.fec44e411cc49p-1, 0x1.fec2ec383a1fap-1, 0x1.fec18a304ce05p-1, 0x1.fec028295505fp-1,
    0x1.febec623528fcp-1, 0x1.febd641e457d4p-1, 0x1.febc021a2dcdbp-1, 0x1.febaa0170b805p-1,
    0x1.feb93e14de94ap-1, 0x1.feb7dc13a709ep-1, 0x1.feb67a1364df6p-1, 0x1.feb5181418149p-1,
    0x1.feb3b615c0a8ap-1, 0x1.feb254185e9b0p-1, 0x1.feb0f21bf1eb0p-1, 0x1.feaf90207a980p-1,
    0x1.feae2e25f8a14p-1, 0x1.feaccc2c6c062p-1, 0x1.feab6a33d4c60p-1, 0x1.feaa083c32e02p-1,
    0x1.fea8a6458653fp-1, 0x1.fea7444fcf20bp-1, 0x1.fea5e25b0d45dp-1, 0x1.fea4806740c28p-1,
    0x1.fea31e7469964p-1, 0x1.fea1bc8287c04p-1, 0x1.fea05a919b3ffp-1, 0x1.fe9ef8a1a4149p-1,
};

// x / 2^40 for |x| < 2^52, exactly (bit assembly instead of an int -> double conversion)
__device__ __forceinline__ double fixed40_to_double(long long x) {
  if (x == 0) return 0.0;
  const unsigned long long neg = x < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int lz = __clzll((long long)a);
  const unsigned long long mant = ((a << lz) << 1) >> 12;  // the bits below the leading one
  const unsigned long long ex = (unsigned long long)(63 - lz - 40 + 1023);
  return __longlong_as_double((long long)(neg | (ex << 52) | mant));
}

// 2^-m T1[a] T2[b] (1 + q) for n = 2^16 m + 2^8 a + b and the remainder r (|r| <= 1/2)
__device__ __forceinline__ double exp2_neg_tail(unsigned long long n, double r) {
  const double q = r * fma(r, kExpC2, -kExpC1);
  const double t2 = __ldg(&kExpT2[n & 255]);
  const double t1 = __ldg(&kExpT1[(n >> 8) & 255]);
  const double v = t1 * fma(t2, q, t2);
  return __longlong_as_double(__double_as_longlong(v) - (long long)((n >> 16) << 52));
}

// 2^(-e / 2^16) for 0 <= e < 2^22
__device__ __forceinline__ double exp2_neg_q16(double e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(e);
  const int u = (int)(b >> 52) - 1023;  // e >= 0: biased exponent only
  unsigned long long n = 0;
  double r = e;  // e < 1/2: n = 0, r = e
  if (u >= -1) {
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int s = u - 12;  // e * 2^40 = M * 2^(u - 12), u - 12 in [-13, 9]
    const unsigned long long F = s >= 0 ? (M << s) : (M >> (-s));
    n = (F + (1ull << 39)) >> 40;
    r = fixed40_to_double((long long)(F - (n << 40)));
  }
  return exp2_neg_tail(n, r);
}

// the same for an argument given in fixed point, F = e 2^40 (0 <= e < 2^22): 4 FP64 operations in all
__device__ __forceinline__ double exp2_neg_fixed40(unsigned long long F) {
  const unsigned long long n = (F + (1ull << 39)) >> 40;
  return exp2_neg_tail(n, fixed40_to_double((long long)(F - (n << 40))));
}

// (a - b)^2 / 2^40 for fixed-point values with |a - b| < 2^52, truncated (at most 2 units below the exact
// quotient), in integer arithmetic: with |a - b| = h 2^32 + l, three 32 x 32 -> 64-bit products
__device__ __forceinline__ unsigned long long sqdiff40(long long a, long long b) {
  const long long d = a - b;
  const unsigned long long u = d < 0 ? (unsigned long long)(-d) : (unsigned long long)d;
  const unsigned h = (unsigned)(u >> 32), l = (unsigned)u;  // h < 2^20
  const unsigned long long hh = (unsigned long long)h * h, hl = (unsigned long long)h * l,
                           ll = (unsigned long long)l * l;
  return (hh << 24) + (hl >> 7) + (ll >> 40);
}

// binary64 -> binary32, round to nearest even, values below FLT_MIN flushed to (signed) zero
__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  unsigned int f = ((unsigned int)e << 23) | (unsigned int)(mant >> 29);
  const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFu);
  f += (rem > 0x10000000u || (rem == 0x10000000u && (f & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | f);
}

// binary32 -> binary64 for normal numbers and zero (subnormals read as zero), exact
__device__ __forceinline__ double f2d_bits(float v) {
  const unsigned int b = __float_as_uint(v);
  const unsigned int ex = (b >> 23) & 0xffu;
  const unsigned long long s = (unsigned long long)(b & 0x80000000u) << 32;
  if (ex == 0) return __longlong_as_double((long long)s);
  return __longlong_as_double((long long)(s | ((unsigned long long)(ex - 127 + 1023) << 52) |
                                          ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// 1/sqrt(d) for a normal d > 0 to about half an ulp, without FP64 instructions (each costs an SM as much
// FP64 pipe time as 32 lanes of work, whatever the number of active lanes).  With d = 4^k d', d' in [1, 4):
// an FP32 seed y0 = rsqrtf(d') (within 2 ulp, so |e| < 2^-21 below), then the second-order correction
// y = y0 (1 + e/2 + 3 e^2 / 8), e = 1 - d' y0^2, whose truncation 5 e^3 / 16 is below 2^-64.  d' = D 2^-52
// and y0 = Y 2^-25 are integers times powers of two, so e is formed exactly in 128-bit integer arithmetic
// (e 2^76, truncated), the correction in fixed point, and the product is rounded to 53 bits.
__device__ __forceinline__ double rsqrt_pivot(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int t = (int)((b >> 52) & 0x7ff) - 1023;
  const int k = t >> 1, sh = t - 2 * k;  // d = 4^k d', d' = 2^sh 1.f
  const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;
  const unsigned long long D = (frac | (1ull << 52)) << sh;
  const double dp = __longlong_as_double((long long)(frac | ((unsigned long long)(1023 + sh) << 52)));
  const unsigned yb = __float_as_uint(rsqrtf(d2f_bits(dp)));
  const int ye = (int)((yb >> 23) & 0xffu) - 127;                                        // -2, -1 or 0
  const unsigned long long Y = (unsigned long long)((yb & 0x7fffffu) | 0x800000u) << (ye + 2);  // y0 = Y 2^-25
  const unsigned long long Y2 = Y * Y;
  const unsigned long long plo = D * Y2, phi = __umul64hi(D, Y2);  // D Y^2 = d' y0^2 2^102
  // e 2^102 = 2^102 - D Y^2 (128-bit), then E = e 2^76
  const unsigned long long qlo = 0ull - plo, qhi = (1ull << 38) - phi - (plo != 0ull ? 1ull : 0ull);
  const long long E = (long long)((qhi << 38) | (qlo >> 26));
  const unsigned long long u = E < 0 ? (unsigned long long)(-E) : (unsigned long long)E;
  const long long e2 = (long long)(__umul64hi(u, u) >> 12);  // e^2 2^76
  const long long dl = (E >> 1) + ((3 * e2) >> 3);          // (e/2 + 3 e^2 / 8) 2^76
  const unsigned long long w = dl < 0 ? (unsigned long long)(-dl) : (unsigned long long)dl;
  unsigned long long zlo = Y * w, zhi = __umul64hi(Y, w);
  if (dl < 0) {
    zhi = ~zhi + (zlo == 0ull ? 1ull : 0ull);
    zlo = 0ull - zlo;
  }
  zhi += Y << 12;  // Z = Y (2^76 + dl) = y 2^(101 + k), Z in (2^100, 2^102)
  const int p = 63 - __clzll((long long)zhi) + 64;
  const int s = p - 52;  // 48 or 49
  unsigned long long mant = (zhi << (64 - s)) | (zlo >> s);
  mant += (zlo >> (s - 1)) & 1ull;  // round half up
  int ex = p - 101 - k;
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  return __longlong_as_double((long long)(((unsigned long long)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace ksdf
