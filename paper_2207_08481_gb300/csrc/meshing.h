// Host-side mesh, dof maps, facet colouring and multigrid hierarchy of libmcs.
#pragma once
#include <cstdint>
#include <vector>

#include "reference.h"

namespace mcs {

struct HostMesh {
  int d = 0;
  int64_t nv = 0, ne = 0;
  std::vector<double> coords;        // [nv][d]
  std::vector<int32_t> elems;        // [ne][d+1] ascending ids
  // facets
  int64_t nf = 0, nint = 0;
  std::vector<int32_t> facets;       // [nf][d] sorted vertex ids, lexicographic
  std::vector<int32_t> elem_facets;  // [ne][d+1]
  std::vector<int32_t> facet_elems;  // [nf][2] (second -1 on the boundary)
  std::vector<int32_t> int_rank;     // [nf] interior rank or -1
  std::vector<int32_t> int_facets;   // [nint] facet id of each interior rank
  std::vector<int8_t> signs;         // [ne][d+1] orientation s_{T,f}
  std::vector<int32_t> elem_rank;    // [ne][d+1] interior rank of local facet f or -1
  std::vector<double> normals;       // [nf][d]
  std::vector<int32_t> int_local;    // [nint][2] local facet index in facet_elems[.][0/1] (-1: none)
  // Gamma_Ntilde (outflow): empty for all-Dirichlet meshes.  When marked, the "interior" ranks above
  // run over the coupling facets, i.e. the interior facets and the outflow facets (facet order).
  std::vector<int8_t> outflow;       // [nf] 1 on Gamma_Ntilde
};

// Builds the facet structures of a mesh with ascending element vertex ids.
void build_facets(HostMesh& m);
// Marks the boundary facets on the face x_1 = 1 as Gamma_Ntilde and renumbers the coupling facets
// (interior and outflow, facet order): int_rank, int_facets, nint, elem_rank, int_local.
void mark_outflow(HostMesh& m);
// C of the tangential penalty of Lemma outflow.
constexpr double kOutflowC = 4.0;
// Kuhn triangulation of [0,1]^d with N cells per direction (dof contract).
HostMesh structured_mesh(int d, int N);

// Greedy facet colouring (interior-facet rank order); returns colour per interior rank.
std::vector<int32_t> colour_facets(const HostMesh& m, int* ncolours);

// Conforming P1 vector space on interior vertices (rank*d + component)
struct P1Space {
  std::vector<int32_t> vrank;  // [nv] interior rank or -1
  int64_t n = 0;               // interior vertices
};
P1Space p1_space(const HostMesh& m);

// CSR matrix (host, FP64)
struct Csr {
  int64_t nrows = 0, ncols = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

// nu (eps u, eps v) on P1 vector fields vanishing on the Dirichlet boundary; with Gamma_Ntilde marked,
// plus the tangential penalty nu C k^2 / h_F int_F u_t . v_t of Lemma outflow (h_F: facet diameter).
Csr abar_matrix(const HostMesh& m, const P1Space& p, double nu, int k = 0);
// P1 interpolation from the N/2 Kuhn mesh to the N mesh (structured hierarchy).
Csr prolongation(int d, int Nc, const P1Space& pc, const P1Space& pf);
Csr transpose(const Csr& A);

// E^d blocks per interior facet: [nint][mF][d*d] (columns: facet vertex w, component a)
std::vector<double> embedding_blocks(const HostMesh& m, const RefTables& T);

}  // namespace mcs
