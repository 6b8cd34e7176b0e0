// Arguments of the GPU assembly kernels (see mm_assemble.cu).
#pragma once
#include <cstdint>

namespace mm {

struct AssembleArgs {
    int nm, nphi;
    double Mref;
    const int* tets;            // [nt][4]
    const int* region;          // [nt]
    const double* materials;    // [nregions][6], SI
    const double* vol;          // [nt] nm^3
    const double* grad;         // [nt][4][3] 1/nm
    const long long* nt_ptr;    // node -> incident tets (ascending)
    const int* nt_idx;
    const int* mag_of;          // node -> magnetic index or -1
    const int* phi_of;          // node -> potential index or -1
    const int* mag_nodes;       // magnetic index -> node
    const int* node_of_phi;     // potential index -> node
    const unsigned char* phi_ident;   // identity row (magnetic node on the outer surface)
    const long long* m_sptr;
    const int* m_col;
    long long nnzm;
    double* KA;
    double* G;
    double* B;
    double* CK;
    double* w;
    double* dinvA;
    const long long* p_sptr;
    const int* p_col;
    double* Kp;
    double* dinvP;
    int* bad;
};

__global__ void k_tet_geometry(int64_t nt, const double* xyz, const int* tets, double* vol,
                               double* grad, int* bad);
__global__ void k_assemble_phi(AssembleArgs A);
__global__ void k_assemble_mag(AssembleArgs A);

}  // namespace mm
