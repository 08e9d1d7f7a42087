/* A caller of the KLB library in plain C: size, allocate, create, step and
 * observe a lattice through the C ABI (include/klb.h) with the CUDA runtime
 * for the device buffer and the stream; no Python, no PyTorch.
 *
 * usage: c_abi_demo nx ny nz radius shell steps tau_w Gx g_we g_wp g_ep g_ec g_pc storage
 * Prints the observables as exact hexadecimal doubles, one "name value" per
 * line; exits non-zero with the library's message on any error. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "klb.h"

static int die(const char *what, const char *msg)
{
    fprintf(stderr, "%s: %s\n", what, msg ? msg : "");
    return 1;
}

int main(int argc, char **argv)
{
    if (argc != 15) return die("usage", "nx ny nz radius shell steps tau_w Gx g_we g_wp g_ep g_ec g_pc storage");
    klb_desc d = {0};
    d.kind = KLB_D3Q19;
    d.nx = atoi(argv[1]);
    d.ny = atoi(argv[2]);
    d.nz = atoi(argv[3]);
    d.geom = KLB_GEOM_PIPE;
    d.radius = atoi(argv[4]);
    d.shell = atoi(argv[5]);
    const long steps = atol(argv[6]);
    d.tau_w = atof(argv[7]);
    d.tau_e = 0.6;
    d.tau_p = 1.0;
    d.rho0 = 1.0;
    d.G[0] = atof(argv[8]);
    d.storage = atoi(argv[14]);
    d.iface_bc = KLB_IFACE_SPECULAR;
    const klb_couplings c = {atof(argv[9]), atof(argv[10]), atof(argv[11]), atof(argv[12]), atof(argv[13])};

    const size_t bytes = klb_lattice_bytes(&d);
    if (!bytes) return die("klb_lattice_bytes", "description rejected");
    void *buf = NULL;
    cudaStream_t stream;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return die("cudaMalloc", "");
    if (cudaStreamCreate(&stream) != cudaSuccess) return die("cudaStreamCreate", "");
    klb_lattice *lat = NULL;
    if (klb_create_lattice(&d, buf, bytes, (void *)stream, &lat) != KLB_OK)
        return die("klb_create_lattice", klb_last_error(NULL));
    if (klb_set_couplings(lat, &c) != KLB_OK) return die("klb_set_couplings", klb_last_error(lat));
    if (klb_step(lat, steps) != KLB_OK) return die("klb_step", klb_last_error(lat));
    klb_obs o;
    if (klb_observables(lat, &o) != KLB_OK) return die("klb_observables", klb_last_error(lat));
    printf("step %lld\n", (long long)o.step);
    printf("flow_rate %a\nslip_length %a\nu_slip %a\nresidual %a\n", o.flow_rate, o.slip_length, o.u_slip,
           o.residual);
    for (int s = 0; s < 3; ++s) printf("mean_u%d %a\nmass%d %a\n", s, o.mean_u[s], s, o.mass[s]);
    if (klb_destroy(lat) != KLB_OK) return die("klb_destroy", klb_last_error(NULL));
    cudaStreamDestroy(stream);
    cudaFree(buf);
    return 0;
}
